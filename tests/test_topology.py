"""The library's topology code (csrc/topology.h), compiled for the host:
which solver fits a scene and the orders that solver relies on.  Checked
against the oracle's own classification (oracle/mabd_oracle.c, written
separately) and against the properties each order must have:

- chain: every free body once, neighbours in the path joined by a joint,
  the two joints of a body next to each other in the joint order (so the
  dual is block tridiagonal, Eq. chain-btd);
- forest: breadth-first levels as ranges, each parent before its children
  and one level up, the parent joint joining the two, the side flag naming
  the child's end, every body's children a contiguous range, a root's
  one-sided joints listed with it (at most two, Sec. 5.3);
- single loop: joint p joins bodies p and p + 1 around the cycle, a ball
  joint as the breaker when there is one (Sec. 5.4);
- every joint exactly once in each order."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2603_08079_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def topo(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path_factory.mktemp("topo") / "topology_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2603_08079_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "topology_check.cpp"), "-o", str(exe)], check=True)

    def run(sc):
        M, K = len(sc["mass"]), len(sc["jtype"])
        lines = [f"{M} {K}", " ".join(str(int(f)) for f in sc["fixed"])]
        lines += [f"{int(a)} {int(b)} {int(t)}" for a, b, t in zip(sc["body_a"], sc["body_b"], sc["jtype"])]
        r = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = {}
        for line in r.stdout.splitlines():
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
        return out
    return run


def _fix_middle(sc):
    sc = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["fixed"][len(sc["fixed"]) // 2] = 1
    return sc


SCENES = {
    "chain_cubes": lambda: scenes.chain_cubes(10),
    "long_chain": lambda: scenes.long_chain(40, seed=2),
    "chain_small": lambda: scenes.random_small("chain", 12, seed=3),
    "chain_unpinned": lambda: scenes.random_small("chain", 9, seed=4, pin=False),
    "chain_fixed_middle": lambda: _fix_middle(scenes.random_small("chain", 11, seed=5)),
    "tree": lambda: scenes.random_tree(200, seed=2, joint="mixed"),
    "assemblies": lambda: scenes.assemblies(10, seed=3),
    "forest": lambda: scenes.random_small("free", 15, seed=6),
    "ring": lambda: scenes.ring_chain(20, seed=1),
    "loop_small": lambda: scenes.random_small("loop", 12, seed=7, pin=False),
    "loop_pinned": lambda: scenes.random_small("loop", 12, seed=7),
    "net": lambda: scenes.jittered_net(4, 4, 3, seed=4),
    "graph": lambda: scenes.random_small("graph", 20, seed=8, univ_frac=0.3, prism_frac=0.3),
}


def _free_joint_ends(sc):
    fixed = np.asarray(sc["fixed"]) != 0
    ends = []
    for a, b in zip(sc["body_a"], sc["body_b"]):
        ends.append(tuple(x for x in (int(a), int(b)) if x >= 0 and not fixed[x]))
    return ends


@pytest.mark.parametrize("name", sorted(SCENES))
def test_classification_matches_the_oracle(ora, topo, name):
    sc = SCENES[name]()
    out = topo(sc)
    o = ora.topology(ora.Scene(sc))  # 1 chain, 2 tree or forest, 3 graph
    assert o in (1, 2, 3)
    if o == 1:
        assert out["chain"] == [1]
    elif o == 2:
        assert out["chain"] == [0] and out["tree"] == [1]
    else:
        assert out["chain"] == [0] and out["tree"] == [0]
    if name in ("ring", "loop_small"):
        assert out["ring"] == [1]
    if name in ("net", "graph"):
        assert out["ring"] == [0]


@pytest.mark.parametrize("name", sorted(SCENES))
def test_orders_have_their_properties(topo, name):
    sc = SCENES[name]()
    out = topo(sc)
    M, K = len(sc["mass"]), len(sc["jtype"])
    fixed = np.asarray(sc["fixed"]) != 0
    free = set(np.flatnonzero(~fixed).tolist())
    nfree = len(free)
    ends = _free_joint_ends(sc)
    if out["chain"] == [1]:
        border, jorder = out["chain_border"], out["chain_jorder"]
        assert sorted(jorder) == list(range(K))
        assert set(border[:nfree]) == free and sorted(border) == list(range(M))
        pos = {k: i for i, k in enumerate(jorder)}
        internal = {frozenset(e) for e in ends if len(e) == 2}
        for u, v in zip(border[:nfree - 1], border[1:nfree]):
            assert frozenset((u, v)) in internal
        for j in free:
            inc = [k for k, e in enumerate(ends) if j in e]
            assert len(inc) <= 2
            if len(inc) == 2:
                assert abs(pos[inc[0]] - pos[inc[1]]) == 1
    if out["tree"] == [1]:
        border, jorder = out["tree_border"], out["tree_jorder"]
        lvl, par, pj, ps = out["tree_lvl"], out["tree_parent"], out["tree_pjoint"], out["tree_pside"]
        cf, cc = out["tree_cfirst"], out["tree_ccount"]
        nr = out["tree_nroots"][0]
        rj, rs = out["tree_rootjoint"], out["tree_rootside"]
        assert sorted(jorder) == list(range(K))
        assert set(border[:nfree]) == free and sorted(border) == list(range(M))
        assert lvl[0] == 0 and lvl[-1] == nfree and all(x < y for x, y in zip(lvl, lvl[1:]))
        level = np.zeros(nfree, dtype=int)
        for d in range(len(lvl) - 1):
            level[lvl[d]:lvl[d + 1]] = d
        roots = 0
        for i in range(nfree):
            if par[i] < 0:
                assert level[i] == 0
                roots += 1
                continue
            p = par[i]
            assert p < i and level[p] == level[i] - 1
            k = pj[i]
            assert set(ends[k]) == {border[i], border[p]}
            assert ps[i] == (0 if int(sc["body_a"][k]) == border[i] else 1)
        assert roots == nr
        for p in range(nfree):
            kids = [i for i in range(nfree) if par[i] == p]
            assert cc[p] == len(kids)
            if kids:
                assert kids == list(range(cf[p], cf[p] + cc[p]))
        # a root's one-sided joints, with the side of the root
        rid = 0
        for i in range(nfree):
            if par[i] >= 0:
                continue
            j = border[i]
            side = sorted(k for k, e in enumerate(ends) if e == (j,))
            got = [rj[w * nr + rid] for w in range(2) if rj[w * nr + rid] >= 0]
            assert got == side
            for w, k in enumerate(got):
                assert rs[w * nr + rid] == (0 if int(sc["body_a"][k]) == j else 1)
            rid += 1
    if out["ring"] == [1]:
        border, jorder = out["ring_border"], out["ring_jorder"]
        assert sorted(jorder) == list(range(K)) and len(border[:nfree]) == K
        for p, k in enumerate(jorder):
            assert set(ends[k]) == {border[p], border[(p + 1) % K]}
        if np.any(np.asarray(sc["jtype"]) == 0):
            assert int(sc["jtype"][jorder[-1]]) == 0
