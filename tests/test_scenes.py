"""The workload generators (paper_2603_08079_gb300/scenes.py) against the
input recipes they state, at reduced sizes: every workload starts
assembled (each joint's constraint C(q_0) = 0, evaluated by the oracle),
at rest in rigid poses, with the stated size, density and joint-type
distributions and the topology its solver expects."""
import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes


def max_gap(ora, sc, q=None):
    S = ora.Scene(sc)
    q = sc["q"] if q is None else q
    return max(float(np.abs(ora.joint_eval(S, q, k)[0]).max()) for k in range(len(sc["jtype"])))


def rigid_rest(sc):
    A = sc["q"][:, :9].reshape(-1, 3, 3).transpose(0, 2, 1)  # columns stacked
    eye = np.einsum("nij,nkj->nik", A, A)
    assert np.abs(eye - np.eye(3)).max() < 1e-12
    assert np.all(np.linalg.det(A) > 0.999)
    assert np.abs(sc["qdot"]).max() == 0.0


def box_sides(sc):
    """Box sides from the diagonal second moments (Sigma_ii = m a_i^2 / 12)."""
    return np.sqrt(12.0 * sc["second_moment"][:, :3] / sc["mass"][:, None])


@pytest.mark.parametrize("name", ["chain_cubes", "long_chain", "ring_chain", "random_tree",
                                  "assemblies", "jittered_net"])
def test_workloads_start_assembled_and_at_rest(ora, name):
    sc = {"chain_cubes": lambda: scenes.chain_cubes(64),
          "long_chain": lambda: scenes.long_chain(3000, seed=1),
          "ring_chain": lambda: scenes.ring_chain(300, seed=1),
          "random_tree": lambda: scenes.random_tree(3000, seed=2),
          "assemblies": lambda: scenes.assemblies(24, seed=3),
          "jittered_net": lambda: scenes.jittered_net(8, 8, 4, seed=4)}[name]()
    rigid_rest(sc)
    scale = float(np.abs(sc["q"][:, 9:]).max()) + 1.0
    assert max_gap(ora, sc) <= 1e-12 * scale
    want = {"chain_cubes": 1, "long_chain": 1, "ring_chain": 3, "random_tree": 2, "assemblies": 2,
            "jittered_net": 3}[name]
    assert ora.topology(ora.Scene(sc)) == want


def test_long_chain_recipe():
    M = 4001
    sc = scenes.long_chain(M, seed=1)
    sides = box_sides(sc)
    rho = sc["mass"] / sc["volume"]
    assert sides.min() >= 0.5 - 1e-12 and sides.max() <= 1.5 + 1e-12
    assert rho.min() >= 1e2 * (1 - 1e-12) and rho.max() <= 1e4 * (1 + 1e-12)
    assert abs(np.log10(rho).mean() - 3.0) < 0.05  # 10^U[2,4]
    K = len(sc["jtype"])
    assert K == M + 1 and sc["body_b"][0] == scenes.WORLD and sc["body_b"][K - 1] == scenes.WORLD
    internal = sc["jtype"][1:K - 1]
    assert np.all(internal[0::2] == scenes.BALL) and np.all(internal[1::2] == scenes.HINGE)
    axes = sc["axis_a"][1:K - 1][1::2]
    assert np.abs(np.linalg.norm(axes, axis=1) - 1.0).max() < 1e-12
    assert np.abs(axes.mean(axis=0)).max() < 0.1  # uniform on the sphere


def test_random_tree_recipe():
    M = 20000
    sc = scenes.random_tree(M, seed=2)
    sides = box_sides(sc)
    assert sides.min() >= 0.2 - 1e-12 and sides.max() <= 1.0 + 1e-12
    assert np.allclose(sc["mass"] / sc["volume"], 1000.0)
    K = len(sc["jtype"])
    assert K == M and sc["body_b"][0] == scenes.WORLD and sc["jtype"][0] == scenes.BALL
    assert np.all(sc["jtype"][1:] == scenes.HINGE)
    parent = sc["body_a"][1:]
    assert np.all(parent < np.arange(1, M))  # creation (BFS) order
    kids = np.bincount(parent, minlength=M)
    inner = kids[:np.max(parent) + 1]
    assert abs(inner.mean() - 1.8) < 0.1  # Poisson(1.8) children of the grown bodies


def test_jittered_net_recipe():
    nx, ny, nz = 12, 10, 6
    sc = scenes.jittered_net(nx, ny, nz, seed=4)
    M = nx * ny * nz
    assert len(sc["mass"]) == M and np.allclose(sc["mass"], 1000.0)
    fixed = sc["fixed"] != 0
    assert fixed.sum() == nx * ny and np.all(fixed[:nx * ny])
    assert np.all(sc["jtype"] == scenes.BALL)
    cand = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    both_fixed = (nx - 1) * ny + nx * (ny - 1)  # bottom-layer pairs, dropped
    n = cand - both_fixed
    K = len(sc["jtype"])
    assert abs(K - 0.7 * n) < 4.0 * np.sqrt(n * 0.21)  # binomial(n, 0.7)
    jitter = sc["q"][:, 9:] - np.round(sc["q"][:, 9:])
    assert abs(jitter.std() - 0.05) < 0.005


def test_assemblies_recipe():
    sc = scenes.assemblies(60, seed=3)
    fixed = np.flatnonzero(sc["fixed"] != 0)
    assert len(fixed) == 60
    sizes = np.diff(np.concatenate([fixed, [len(sc["mass"])]]))
    assert sizes.min() >= 7 and sizes.max() <= 64
    free = sc["fixed"] == 0
    assert sc["mass"][free].min() >= 0.1 * (1 - 1e-12) and sc["mass"][free].max() <= 10.0 * (1 + 1e-12)
    sides = box_sides(sc)[free]
    assert sides.min() >= 0.1 - 1e-12 and sides.max() <= 0.5 + 1e-12
    frac_hinge = float(np.mean(sc["jtype"] == scenes.HINGE))
    assert abs(frac_hinge - 0.5) < 0.1
