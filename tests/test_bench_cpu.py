"""Host-side pieces of the benchmark: the batch's assemblies split into
scenes of their own give, step by step, the oracle's result on the whole
batch (they are independent), and the all-core oracle baseline runs them in
spawned worker processes."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_split_assemblies_matches_the_whole_batch(ora):
    import bench
    from paper_2603_08079_gb300 import scenes
    sc = scenes.assemblies(6, seed=3)
    q, qd = scenes.perturb_state(sc, seed=1, rot=0.05, vel=0.3)
    full = dict(sc, q=q, qdot=qd)
    q1, qd1, lam, _ = ora.step(ora.Scene(full), q, qd)
    subs = bench.split_assemblies(full)
    assert len(subs) == 6 and sum(len(s["mass"]) for s in subs) == len(sc["mass"])
    assert sum(len(s["jtype"]) for s in subs) == len(sc["jtype"])
    parts_q, parts_qd, parts_lam = [], [], []
    for s in subs:
        a, b, l, _ = ora.step(ora.Scene(s), s["q"], s["qdot"])
        parts_q.append(a)
        parts_qd.append(b)
        parts_lam.append(l)
    np.testing.assert_allclose(np.concatenate(parts_qd), qd1, rtol=0, atol=1e-12 * np.max(np.abs(qd1)))
    np.testing.assert_allclose(np.concatenate(parts_q), q1, rtol=0, atol=1e-12 * np.max(np.abs(q1)))
    np.testing.assert_allclose(np.concatenate(parts_lam), lam, rtol=0, atol=1e-10 * np.max(np.abs(lam)))


def test_parallel_oracle_baseline_runs():
    import bench
    bodies, dt, cores = bench.batch_oracle_parallel(1, 1, n=16, seed=3)
    from paper_2603_08079_gb300 import scenes
    assert bodies == len(scenes.assemblies(16, seed=3)["mass"])
    assert dt > 0 and cores >= 1


def test_roofline_byte_models_by_hand():
    """The algorithmic-bytes models behind the bench line's roofline, against
    hand counts on tiny chains: the residual kernel (per body 476 B, per ball
    joint 73 B, per hinge joint 209 B, 10 B of incidence per joint) and the
    back-substitution of a 3-row chain of two levels."""
    import bench
    from paper_2603_08079_gb300 import scenes
    jt = np.array([0, 1, 0, 1, 0])          # 4 bodies, ball/hinge alternating
    assert bench.mx_res_body_bytes(jt, 4) == 4 * 476 + 3 * 73 + 2 * 209 + 5 * 10
    assert list(scenes.joint_rows([0, 1, 2, 3])) == [3, 5, 4, 5]
    # three ball rows: one level eliminates row 1 (neighbours 0 and 2) and
    # keeps rows 0, 2; the next level eliminates row 1 of (0, 2) with only a
    # left neighbour (FP32 records, level 0 writes FP64 multipliers)
    # (the odd row reads its factor record n(n+1)/2 + n l + n r + n and its
    # neighbours' l + r multipliers and writes n; each even row copies n)
    balls = np.zeros(3, dtype=np.int64)
    assert bench._cr_sizes(balls).tolist() == [3, 3, 3]
    first = (6 + 9 + 9 + 3 + 3 + 3) * 4 + 3 * 8 + 2 * 3 * (4 + 8)
    second = (6 + 9 + 0 + 3 + 3 + 0) * 4 + 3 * 4 + 1 * 3 * (4 + 4)
    assert bench.cr_back_bytes(balls, 4) == first + second


def test_normalized_pcg_byte_model_and_graph_entries(ora):
    """The joint graph's entry count used by the net's roofline equals the
    oracle's joint graph (ordered pairs of joints sharing a free body), and
    the per-iteration byte model adds up its per-joint and per-entry terms
    (232 B per joint, 132 B per stored block on average)."""
    import bench
    from oracle import lpc
    from paper_2603_08079_gb300 import scenes
    sc = scenes.jittered_net(5, 4, 3, seed=7)
    ent, ones = lpc.joint_graph(sc)
    nnz = sum(len(e) for e in ent)
    assert bench.joint_graph_entries(sc) == nnz
    K = len(sc["jtype"])
    assert bench.pcgn_iteration_bytes(K, nnz) == K * 232 + nnz * 132


def test_reference_arm_line_keeps_the_contract():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys of the benchmark contract, on a small sample."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-bodies", "2048"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "body-steps/s"
    assert d["steps"] == 1 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
