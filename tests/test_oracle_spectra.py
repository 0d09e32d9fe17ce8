"""The spectral report's dual operator against the dense KKT pieces of the
oracle (assemble_dense): the same S = G H^{-1} G^T on small scenes of every
topology, and Lanczos extremes against dense eigenvalues."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes


def dense_from_assembly(ora, sc, q, qd):
    S_ = ora.Scene(sc)
    Hw, f, G, c = ora.assemble_dense(S_, q, qd)
    n = G.shape[0]
    S = np.zeros((n, n))
    fixed = np.asarray(sc["fixed"]) != 0
    for j in range(len(sc["mass"])):
        if fixed[j]:
            continue
        Gj = G[:, 12 * j:12 * j + 12]
        S += Gj @ np.linalg.solve(Hw[j], Gj.T)
    return 0.5 * (S + S.T)


@pytest.mark.parametrize("case", ["chain", "tree", "net", "loop"])
def test_operator_matches_dense_assembly(ora, case):
    from oracle import spectra
    sc = {"chain": lambda: scenes.long_chain(9, seed=1), "tree": lambda: scenes.random_small("tree", 8, seed=2),
          "net": lambda: scenes.jittered_net(3, 3, 2, seed=4),
          "loop": lambda: scenes.random_small("loop", 7, seed=3)}[case]()
    q, qd = scenes.perturb_state(sc, seed=5, rot=0.3, vel=0.2)
    S = spectra.dense_dual(sc, q, qd)
    Sd = dense_from_assembly(ora, sc, q, qd)
    assert np.abs(S - Sd).max() <= 1e-9 * np.abs(Sd).max()


def test_lanczos_extremes_match_dense_eigenvalues(ora):
    from oracle import spectra
    sc = scenes.jittered_net(3, 3, 2, seed=4)
    n, apply = spectra.dual_operator(sc)
    w = np.linalg.eigvalsh(spectra.dense_dual(sc))
    lo, hi, rlo, rhi, m = spectra.lanczos(apply, n, steps=4 * n)
    assert abs(hi - w[-1]) <= 1e-8 * w[-1]
    assert abs(lo - w[0]) <= 1e-6 * w[-1]
