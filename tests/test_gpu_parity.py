"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Bar (labels): bit-exact at every iteration except objects whose FP64 top-2
margin is below 1e-6 (counted). Centroids: same sparsity pattern, values
within 1e-5 relative. Objectives: within 1e-6 relative.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import Oracle
from synth import CONFIGS, generate, init_ids
from synth.corpus import from_dense
from tests.gpu_harness import (compare_centroids, compare_labels, corpus_for, gpu_instance, lockstep, rel,
                               OBJECTIVE_RTOL)
from tests.helpers import random_dense_corpus

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("update_mode", ["dense", "sort"])
def test_c1_lockstep_fp32_icp(update_mode):
    w = CONFIGS["c1"]
    c, ini = corpus_for(w)
    recs = lockstep(c, w.k, ini, w.max_iter, update_mode=update_mode)
    assert recs[-1]["changed"] == 0 or len(recs) == w.max_iter
    assert all(r["stats"]["update_dense"] == (update_mode == "dense") for r in recs)


@pytest.mark.parametrize("update_mode", ["dense", "sort"])
def test_update_modes_on_long_lists(update_mode):
    """Both forms of the update step (dense fixed-point accumulator, sorted
    FP64 runs) against the oracle's centroids and objectives."""
    w = CONFIGS["c2"].scaled(N=8_000, D=1_500, k=500, mu=3.5, hi=400)
    c, ini = corpus_for(w, seed=41)
    lockstep(c, w.k, ini, 10, update_mode=update_mode)


@pytest.mark.parametrize("threads", [32, 64, 128, 512])
def test_mid_lockstep_block_sizes(threads):
    # several tiles of objects, documents longer than one staging chunk, ragged tails
    w = CONFIGS["c2"].scaled(N=6_000, D=8_000, k=60, hi=1500)
    c, ini = corpus_for(w, seed=5)
    lockstep(c, w.k, ini, 8, threads=threads)


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_long_lists_tiled_blocks(precision):
    """Posting lists of up to three full 128-entry blocks plus a ragged tail
    (a 1,500-term vocabulary shared by k = 500 centroids), with ICP fronts
    longer than one block that end inside a full block (iterations 3-6): the
    tiled scan layout against the oracle."""
    w = CONFIGS["c2"].scaled(N=8_000, D=1_500, k=500, mu=3.5, hi=400)
    c, ini = corpus_for(w, seed=31)
    recs = lockstep(c, w.k, ini, 10, precision=precision)
    assert any(r["stats"]["filtered"] > 0 for r in recs)


def test_free_running_c1_matches_oracle_every_iteration():
    w = CONFIGS["c1"]
    c, ini = corpus_for(w)
    g = gpu_instance(c, w.k, ini)
    o = Oracle(c, w.k, ini, icp=True)
    ou = Oracle(c, w.k, ini, icp=False)
    try:
        for _ in range(w.max_iter):
            g.assign()
            a = o.assign()
            ou.assign()
            best, second, _ = ou.scores()
            n = compare_labels(g.labels(), o.labels(), best, second, f"iteration {a.r}")
            assert n == 0, "free-running trajectories diverged on a near-tie"
            if a.r > 1 and a.changed == 0:
                break
            g.update()
            u = o.update()
            ou.update()
            assert rel(g.stats()["objective_update"], u.objective) <= OBJECTIVE_RTOL
    finally:
        g.close()


def test_icp_and_unfiltered_gpu_runs_are_bit_identical():
    w = CONFIGS["c2"].scaled(N=8_000, D=10_000, k=80)
    c, ini = corpus_for(w, seed=9)
    f = gpu_instance(c, w.k, ini, icp=True)
    u = gpu_instance(c, w.k, ini, icp=False)
    try:
        saw_filter = False
        for _ in range(25):
            nf, nu = f.assign(), u.assign()
            assert nf == nu
            assert np.array_equal(f.labels(), u.labels())
            assert np.array_equal(f.lam(), u.lam())
            sf, su = f.stats(), u.stats()
            saw_filter |= sf["filtered"] > 0
            assert su["simcalc"] == w.N * w.k
            assert sf["postings"] <= su["postings"]
            if sf["iter"] > 1 and nf == 0:
                break
            f.update()
            u.update()
            cf, cu = f.centroids(), u.centroids()
            for x, y in zip(cf, cu):
                assert np.array_equal(x, y)
            assert f.stats()["objective_update"] == u.stats()["objective_update"]
        assert saw_filter
    finally:
        f.close()
        u.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_mixed_precision_labels_match_oracle(precision):
    w = CONFIGS["c2"].scaled(N=6_000, D=8_000, k=120)
    c, ini = corpus_for(w, seed=13)
    recs = lockstep(c, w.k, ini, 6, precision=precision)
    assert sum(r["stats"]["rescored"] for r in recs) > 0


def test_duplicate_documents_and_seed_ties():
    # identical documents give identical seeds: exact ties broken by lowest index
    X, c = random_dense_corpus(300, 200, 0.05, seed=3, dup_rows=40)
    N = c.N
    ini = np.array([0, N - 1, 5, 7, 11, 13, 17, 19], dtype=np.int32)  # rows 0 and N-1 are identical
    lockstep(c, len(ini), ini, 15)


def test_edge_cases_k1_kN_empty_rows():
    X, c = random_dense_corpus(50, 300, 0.05, seed=4)
    lockstep(c, 1, np.array([3], dtype=np.int32), 5)
    lockstep(c, 50, np.random.default_rng(1).permutation(50).astype(np.int32), 5)
    X = np.zeros((40, 30), dtype=np.float32)
    rng = np.random.default_rng(2)
    for i in range(36):
        m = rng.random(30) < 0.2
        m[rng.integers(30)] = True
        X[i, m] = rng.random(m.sum()) + 0.1
        X[i] /= np.linalg.norm(X[i])
    X[36:, :] = 0.0  # four empty rows: every score is zero, label 0
    lockstep(from_dense(X), 4, np.array([0, 1, 2, 3], dtype=np.int32), 10)


def test_full_size_c2_sampled_against_oracle():
    """The bench workload at full size (N = 300K, D = 100K, k = 1000), in the
    bench's launch configuration: after each assignment a sample of objects is
    scored one by one by the oracle against centroids rebuilt from the GPU's
    own previous labels."""
    w = CONFIGS["c2"]
    c, ini = corpus_for(w)
    g = gpu_instance(c, w.k, ini)
    o = Oracle(c, w.k, ini, icp=False)
    rng = np.random.default_rng(0)
    try:
        for r in range(1, 4):
            g.assign()
            lab = g.labels()
            ids = np.sort(rng.choice(w.N, size=3000, replace=False))
            lab_o, best, second = o.score_objects(ids)
            compare_labels(lab[ids], lab_o, best, second, f"C2 iteration {r}")
            o.set_labels(lab)
            g.update()
            u = o.update()
            assert rel(g.stats()["objective_update"], u.objective) <= OBJECTIVE_RTOL
        compare_centroids(g, o)
    finally:
        g.close()


def _batch_corpora(n_inst, scale, seed0=0):
    from synth import batched_instances, generate, init_ids
    ws = batched_instances(n_inst, scale=scale)
    cs = [generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed + seed0) for w in ws]
    inis = [init_ids(w.N, w.k, w.init_seed) for w in ws]
    return ws, cs, inis


@pytest.mark.parametrize("precision,update_mode", [("fp32", "dense"), ("fp16", "dense"), ("fp32", "sort")])
def test_batched_instances_match_their_own_oracles(precision, update_mode):
    """Several uneven instances in one context: at every iteration each
    instance's labels equal its own FP64 oracle's (near ties excepted)."""
    from paper_2103_16141_gb300 import SIVFBatch
    ws, cs, inis = _batch_corpora(6, scale=0.05)
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision=precision, update_mode=update_mode)
    ors = [Oracle(c, w.k, ini, icp=True) for w, c, ini in zip(ws, cs, inis)]
    ous = [Oracle(c, w.k, ini, icp=False) for w, c, ini in zip(ws, cs, inis)]
    done = [False] * len(ws)
    try:
        for _ in range(30):
            b.assign()
            for m, (o, ou) in enumerate(zip(ors, ous)):
                if done[m]:
                    continue
                a = o.assign()
                ou.assign()
                best, second, _ = ou.scores()
                n = compare_labels(b.labels(m), o.labels(), best, second, f"instance {m} r={a.r}")
                assert n == 0
                assert b.instance_stats(m)["changed"] == a.changed
                if a.r > 1 and a.changed == 0:
                    done[m] = True
            if all(done):
                break
            b.update()
            for m, (o, ou) in enumerate(zip(ors, ous)):
                if done[m]:
                    continue
                u = o.update()
                ou.update()
                assert rel(b.instance_stats(m)["objective_update"], u.objective) <= OBJECTIVE_RTOL
        assert all(done)
    finally:
        b.close()


def test_batched_run_equals_separate_runs():
    """sivf_batch_run gives every instance the labels and iteration count of
    its own single-instance run."""
    from paper_2103_16141_gb300 import SIVFBatch
    ws, cs, inis = _batch_corpora(5, scale=0.04, seed0=100)
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16")
    try:
        iters, obj = b.run(50)
        for m, (w, c, ini) in enumerate(zip(ws, cs, inis)):
            g = gpu_instance(c, w.k, ini, precision="fp16")
            try:
                it1, _ = g.run(50)
                assert np.array_equal(b.labels(m), g.labels())
                assert iters[m] == it1
            finally:
                g.close()
    finally:
        b.close()


@pytest.mark.parametrize("update_mode", ["dense", "sort"])
def test_graph_loop_equals_host_stepped_run(update_mode):
    """With use_graph the iterations after the second run inside one CUDA graph
    (WHILE conditional node): same labels, iteration count, objective and
    centroids as the host-stepped run."""
    w = CONFIGS["c2"].scaled(N=8_000, D=10_000, k=80)
    c, ini = corpus_for(w, seed=17)
    a = gpu_instance(c, w.k, ini, use_graph=False, update_mode=update_mode)
    b = gpu_instance(c, w.k, ini, use_graph=True, update_mode=update_mode)
    try:
        ia, oa = a.run(40)
        ib, ob = b.run(40)
        assert b.stats()["graph_iters"] > 0, b.last_error()
        assert a.stats()["graph_iters"] == 0
        assert ia == ib
        assert np.array_equal(a.labels(), b.labels())
        assert oa == ob
        for x, y in zip(a.centroids(), b.centroids()):
            assert np.array_equal(x, y)
        # a second call continues from the converged state identically
        assert a.run(5)[0] == b.run(5)[0]
        # reseeding reuses the captured graph
        a.reseed(ini)
        b.reseed(ini)
        assert a.run(40) == b.run(40)
        assert np.array_equal(a.labels(), b.labels())
    finally:
        a.close()
        b.close()


def test_graph_loop_batched_equals_host_stepped():
    from paper_2103_16141_gb300 import SIVFBatch
    ws, cs, inis = _batch_corpora(5, scale=0.04, seed0=200)
    a = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", use_graph=False)
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision="fp16", use_graph=True)
    try:
        ia, oa = a.run(50)
        ib, ob = b.run(50)
        assert b.stats()["graph_iters"] > 0, b.last_error()
        assert np.array_equal(ia, ib)
        assert np.array_equal(oa, ob)
        for m in range(len(ws)):
            assert np.array_equal(a.labels(m), b.labels(m))
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("score_buffer", ["global"])
def test_global_score_buffer_matches_oracle(score_buffer):
    w = CONFIGS["c2"].scaled(N=4_000, D=6_000, k=70)
    c, ini = corpus_for(w, seed=23)
    lockstep(c, w.k, ini, 6, score_buffer=score_buffer)


def test_autotuned_run_equals_default_run():
    """The autotuner's trial launches leave no trace: the tuned run produces
    the default run's labels and iteration count."""
    w = CONFIGS["c2"].scaled(N=8_000, D=10_000, k=80)
    c, ini = corpus_for(w, seed=29)
    a = gpu_instance(c, w.k, ini)
    b = gpu_instance(c, w.k, ini, autotune=True)
    try:
        ra, rb = a.run(40), b.run(40)
        assert ra == rb
        assert np.array_equal(a.labels(), b.labels())
        st = b.stats()
        assert st["assign_threads"] in (64, 128, 256, 512)
    finally:
        a.close()
        b.close()


def test_host_inputs_equal_device_inputs():
    """inputs_on_host: the library copies a pinned host CSR itself; the run is
    the same as from borrowed device arrays, and the host arrays may be
    released right after init."""
    import torch
    w = CONFIGS["c2"].scaled(N=6_000, D=8_000, k=90)
    c, ini = corpus_for(w, seed=37)
    a = gpu_instance(c, w.k, ini)
    rp = torch.from_numpy(c.row_ptr.copy()).pin_memory()
    ix = torch.from_numpy(c.idx.copy()).pin_memory()
    vl = torch.from_numpy(c.val.copy()).pin_memory()
    from paper_2103_16141_gb300 import SIVF
    b = SIVF(rp, ix, vl, c.D, w.k, ini, inputs_on_host=True)
    del rp, ix, vl
    try:
        ra, rb = a.run(40), b.run(40)
        assert ra == rb
        assert np.array_equal(a.labels(), b.labels())
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cbicp_lockstep_against_oracle(precision):
    """IVF-CBICP (Algorithm 3) on the GPU against the oracle in the same mode:
    labels, filtered objects, sim-calcs and postings traversed."""
    w = CONFIGS["c2"].scaled(N=8_000, D=1_500, k=500, mu=3.5, hi=400)
    c, ini = corpus_for(w, seed=43)
    recs = lockstep(c, w.k, ini, 10, precision=precision, icp="cbicp")
    assert any(r["stats"]["filtered"] > 0 for r in recs)


def test_cbicp_sivf_ivf_three_way_on_gpu():
    """The three assignment algorithms give the same labels at every
    iteration; CBICP's sim-calcs equal SIVF's and its postings equal IVF's."""
    w = CONFIGS["c2"].scaled(N=8_000, D=10_000, k=80)
    c, ini = corpus_for(w, seed=47)
    s, v, b = (gpu_instance(c, w.k, ini, icp=m) for m in (True, False, "cbicp"))
    try:
        saw_filter = False
        for _ in range(25):
            ns, nv, nb = s.assign(), v.assign(), b.assign()
            assert ns == nv == nb
            assert np.array_equal(s.labels(), v.labels()) and np.array_equal(b.labels(), v.labels())
            ss, sv, sb = s.stats(), v.stats(), b.stats()
            assert sb["simcalc"] == ss["simcalc"] and sb["filtered"] == ss["filtered"]
            assert sb["postings"] == sv["postings"]
            saw_filter |= sb["filtered"] > 0
            if ss["iter"] > 1 and ns == 0:
                break
            s.update(), v.update(), b.update()
        assert saw_filter
    finally:
        for g in (s, v, b):
            g.close()


@pytest.mark.parametrize("precision,case", [("fp32", (3000, 3000, 30, 31)), ("bf16", (2000, 1000, 25, 33)),
                                            ("fp32", (4000, 2000, 20, 31))])
def test_relaxed_filter_lockstep(precision, case):
    """SIVF with the relaxed filter on the GPU: the oracle's labels at every
    iteration, and the objects it restricts to the moving centroids are at
    least SIVF's and at most the oracle's (its test is error-bounded)."""
    N, D, k, seed = case
    w = CONFIGS["c1"].scaled(N=N, D=D, k=k)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, seed)
    ini = init_ids(w.N, w.k, seed)
    recs = lockstep(c, k, ini, 60, precision=precision, icp="relaxed")
    s = gpu_instance(c, k, ini, precision=precision)
    try:
        extra = 0
        for r in recs:
            s.assign()
            extra += r["stats"]["filtered"] - s.stats()["filtered"]
            assert r["stats"]["filtered"] >= s.stats()["filtered"]
            if r["r"] > 1 and r["changed"] == 0:
                break
            s.update()
        assert extra > 0
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp16"])
def test_k_above_65536_uses_32_bit_ids_and_global_scores(precision):
    """k = 66,000 clusters (over the 16-bit id range, and a score vector too
    large for shared memory): 32-bit scan ids (with FP32 values, or 16-bit
    values in their own array) and per-CTA score slabs in global memory,
    against the oracle."""
    c = generate(70_000, 400_000, 0.6, float(np.log(8.0)), 0.3, 5, 16, 77)
    ini = init_ids(c.N, 66_000, 78)
    recs = lockstep(c, 66_000, ini, 3, precision=precision)
    assert recs[0]["stats"]["assign_global"] == 1


@pytest.mark.parametrize("inputs_on_host", [False, True])
def test_device_label_buffers_equal_host_buffers(inputs_on_host):
    """sivf_get_labels and sivf_set_labels with DEVICE buffers give what the
    HOST buffers give: the labels copied into a device tensor equal the host
    copy, and a twin context resynchronised from a device buffer reaches the
    same lambda, centroids and next labels as one resynchronised from the
    host (also for a context built from host inputs)."""
    import torch
    w = CONFIGS["c1"]
    c, ini = corpus_for(w)
    a = gpu_instance(c, w.k, ini, inputs_on_host=inputs_on_host)
    b = gpu_instance(c, w.k, ini, inputs_on_host=inputs_on_host)
    try:
        for s in (a, b):
            s.assign()
            s.update()
            s.assign()
        lab = a.labels()
        dl = a.labels_device()
        assert dl.device == a.device and np.array_equal(dl.cpu().numpy(), lab)
        out = torch.full((c.N,), -7, dtype=torch.int32, device=a.device)
        assert a.labels_device(out) is out and np.array_equal(out.cpu().numpy(), lab)
        moved = ((lab + 1) % w.k).astype(np.int32)  # every object changes cluster
        a.set_labels(moved)
        b.set_labels(torch.from_numpy(moved).to(b.device))
        assert np.array_equal(a.labels(), moved) and np.array_equal(b.labels(), moved)
        assert np.array_equal(a.lam(), b.lam())
        a.update()
        b.update()
        for x, y in zip(a.centroids(), b.centroids()):
            assert np.array_equal(x, y)
        a.assign()
        b.assign()
        assert np.array_equal(a.labels(), b.labels())
    finally:
        a.close()
        b.close()
