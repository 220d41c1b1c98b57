"""Batched independent clients (one multi-client launch per kernel, tau local
steps in a CUDA graph) against the same clients stepped one at a time and
against the FP64 oracle, client by client."""
import math

import numpy as np
import pytest

import oracle
import synth
from adam_readout import flat, readout_params, recover_gradient

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def bf16_round(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def env(gpu_lib):
    import torch

    return gpu_lib, torch


@pytest.fixture(scope="module")
def shards():
    cl = synth.client_batch(7, 5005, dim_lo=40, dim_hi=300, nnz_lo=300, nnz_hi=20000)
    out = []
    for i, (dims, coords, vals) in enumerate(cl):
        f = synth.factors_uniform(dims, 16, 6000 + i, lo=0.1, hi=1.0)
        S = max(1, math.ceil(len(vals) / 8))
        out.append(dict(dims=dims, coords=coords, vals=vals, factors=f, p=S, q=S + 3 * i, seed=7000 + i))
    return out


def make(gcp, shards, dtype="fp32"):
    ctxs = []
    for s in shards:
        c = gcp.gcp_create(s["dims"], s["coords"], s["vals"], 16, "poisson", dtype=dtype, seed=s["seed"])
        c.set_factors(s["factors"])
        ctxs.append(c)
    return ctxs


ADAM = dict(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_batch_matches_clients_stepped_one_at_a_time(env, shards, dtype):
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    ref = make(gcp, shards, dtype)
    for c, s in zip(ref, shards):
        for k in range(3):
            L, _ = c.grad(5 + k, s["p"], s["q"])
            c.adam_step(adam, k + 1)
        s["ref_loss"] = L
    bat = make(gcp, shards, dtype)
    b = gcp.GcpBatch(bat, [s["p"] for s in shards], [s["q"] for s in shards])
    b.local_steps(3, adam, 5, 0)
    losses = b.losses()
    for c, r, s, L in zip(bat, ref, shards, losses):
        A = np.concatenate([a.ravel() for a in c.get_factors()])
        Ar = np.concatenate([a.ravel() for a in r.get_factors()])
        assert rel_err(A, Ar) <= 1e-5
        assert L == pytest.approx(s["ref_loss"], rel=1e-6)
    b.close()


def test_batch_one_step_matches_oracle_client_by_client(env, shards):
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    bat = make(gcp, shards)
    b = gcp.GcpBatch(bat, [s["p"] for s in shards], [s["q"] for s in shards])
    b.local_steps(1, adam, 11, 0)
    losses = b.losses()
    for c, s, L in zip(bat, shards, losses):
        idx, x, w, _ = oracle.stratified_samples(s["seed"], 11, s["p"], s["q"], s["dims"], s["coords"], s["vals"])
        Lo, Go = oracle.sampled_loss_grad(s["dims"], s["factors"], "poisson", idx, x, w)
        A = oracle.flat_factors(s["factors"])
        B, C = np.zeros_like(A), np.zeros_like(A)
        oracle.adam_step(A, B, C, np.concatenate([g.ravel() for g in Go]), **{
            "lr": 1e-3, "beta1": 0.9, "beta2": 0.999, "eps": 1e-8, "lower": 0.0, "t": 1})
        Ag = np.concatenate([a.ravel() for a in c.get_factors()])
        assert L == pytest.approx(Lo, rel=1e-5)
        assert rel_err(Ag, A) <= 1e-5
    b.close()


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
@pytest.mark.parametrize("tile", [16, 32, 64])
def test_batch_folded_gradient_matches_oracle_client_by_client(env, shards, dtype, tile):
    """The gradient each client's local step folds (multi-client fused pass,
    then k_batch_post's replica fold) and feeds to Adam, read back through a
    readout Adam step (tests/adam_readout.py) and compared element by
    element with the oracle's sampled gradient, per client and mode, with
    16, 32 and 64 samples per warp tile.  Every mode of these shards has at
    most 300 rows, so every row is replicated."""
    gcp, torch = env
    bat = make(gcp, shards, dtype)
    ref = []
    for s in shards:
        fac = [bf16_round(a) for a in s["factors"]] if dtype == "bf16" else s["factors"]
        idx, x, w, _ = oracle.stratified_samples(s["seed"], 13, s["p"], s["q"], s["dims"], s["coords"], s["vals"])
        ref.append(oracle.sampled_loss_grad(s["dims"], fac, "poisson", idx, x, w))
    prm = readout_params(gcp, max(np.abs(g).max() for _, Go in ref for g in Go))
    b = gcp.GcpBatch(bat, [s["p"] for s in shards], [s["q"] for s in shards])
    b.tune(samples_per_warp=tile)
    b.local_steps(1, prm, 13, 0)
    losses = b.losses()
    for c, s, (Lo, Go), L in zip(bat, shards, ref, losses):
        G = recover_gradient(flat(s["factors"]), flat(c.get_factors()), prm)
        assert L == pytest.approx(Lo, rel=1e-5)
        o = 0
        for n, g in enumerate(Go):
            assert rel_err(G[o:o + g.size], g) <= 1e-5, (s["seed"], n, rel_err(G[o:o + g.size], g))
            o += g.size
    b.close()


def test_graph_replays_continue_the_step_counters(env, shards):
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    one = make(gcp, shards)
    b1 = gcp.GcpBatch(one, [s["p"] for s in shards], [s["q"] for s in shards])
    b1.local_steps(4, adam, 0, 0)
    two = make(gcp, shards)
    b2 = gcp.GcpBatch(two, [s["p"] for s in shards], [s["q"] for s in shards])
    b2.local_steps(2, adam, 0, 0)
    b2.local_steps(2, adam, 2, 2)  # graph reused, counters reset from the host
    for c1, c2 in zip(one, two):
        a1 = np.concatenate([a.ravel() for a in c1.get_factors()])
        a2 = np.concatenate([a.ravel() for a in c2.get_factors()])
        assert rel_err(a2, a1) <= 1e-5
    b1.close()
    b2.close()


@pytest.mark.parametrize("cols,blocks,tile", [(8, 0, 32), (4, 3, 32), (8, 1, 64), (4, 0, 16), (8, 5, 16), (4, 0, 64)])
def test_tuning_knobs_do_not_change_results(env, shards, cols, blocks, tile):
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    base = make(gcp, shards)
    b0 = gcp.GcpBatch(base, [s["p"] for s in shards], [s["q"] for s in shards])
    b0.local_steps(2, adam, 3, 0)
    tuned = make(gcp, shards)
    b1 = gcp.GcpBatch(tuned, [s["p"] for s in shards], [s["q"] for s in shards])
    b1.tune(cols, blocks, samples_per_warp=tile)
    b1.local_steps(2, adam, 3, 0)
    for c0, c1 in zip(base, tuned):
        a0 = np.concatenate([a.ravel() for a in c0.get_factors()])
        a1 = np.concatenate([a.ravel() for a in c1.get_factors()])
        assert rel_err(a1, a0) <= 1e-5
    b0.close()
    b1.close()


def test_tile_size_knob_rejects_other_sizes_and_switches_back(env, shards):
    """gcp_batch_tune_tile takes 16, 32 or 64 (0 = 32); the graph is rebuilt
    when the size changes, and switching 64 -> 16 -> 32 between calls gives
    the same models as staying at 32 (up to FP32 summation order)."""
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    a = make(gcp, shards)
    ba = gcp.GcpBatch(a, [s["p"] for s in shards], [s["q"] for s in shards])
    for bad in (8, 48, 128, -16):
        with pytest.raises(gcp.GcpError):
            ba.tune(samples_per_warp=bad)
    for k, tile in enumerate((64, 16, 0)):
        ba.tune(samples_per_warp=tile)
        ba.local_steps(1, adam, 20 + k, k)
    r = make(gcp, shards)
    br = gcp.GcpBatch(r, [s["p"] for s in shards], [s["q"] for s in shards])
    br.local_steps(3, adam, 20, 0)
    for c0, c1 in zip(a, r):
        a0 = np.concatenate([x.ravel() for x in c0.get_factors()])
        a1 = np.concatenate([x.ravel() for x in c1.get_factors()])
        assert rel_err(a0, a1) <= 1e-5
    ba.close()
    br.close()


def test_batch_rejects_mismatched_clients(env, shards):
    gcp, torch = env
    s0, s1 = shards[0], shards[1]
    a = gcp.gcp_create(s0["dims"], s0["coords"], s0["vals"], 16, "poisson")
    c = gcp.gcp_create(s1["dims"], s1["coords"], s1["vals"], 8, "poisson")
    with pytest.raises(gcp.GcpError):
        gcp.GcpBatch([a, c], [10, 10], [10, 10])
    with pytest.raises(gcp.GcpError):
        gcp.GcpBatch([a], [-1], [10])
    with pytest.raises(ValueError):
        gcp.GcpBatch([a], [10, 10], [10])  # one count per client


def test_batch_of_64_clients_full_size_against_oracle(env):
    """64 client shards, mode sizes U{200..5000}, nnz log-uniform in
    [1e4, 2e6], 1+Poisson(2), Poisson loss, rank 16, BF16 factors with FP32
    accumulation, p_c = q_c = ceil(nnz_c / 8): one local step of every client
    in one graph launch.  Each client's loss, and the gradient its epilogue
    folds and feeds to Adam (read back through a readout Adam step,
    tests/adam_readout.py), against the oracle on the same samples and the
    same BF16-rounded factors, per client and mode, at 1e-5."""
    gcp, torch = env
    shards = synth.cached("client_batch_64", lambda: synth.client_batch(64, 1005))
    clients, P, facs, ref = [], [], [], []
    for i, (dims, coords, vals) in enumerate(shards):
        c = gcp.gcp_create(dims, coords, vals, 16, "poisson", dtype="bf16", seed=5000 + i)
        f = synth.factors_uniform(dims, 16, 6000 + i, lo=0.1, hi=1.0)
        c.set_factors(f)
        clients.append(c)
        facs.append(f)
        P.append(math.ceil(len(vals) / 8))
        idx, x, w, _ = oracle.stratified_samples(5000 + i, 9, P[i], P[i], dims, coords, vals)
        ref.append(oracle.sampled_loss_grad(dims, [bf16_round(a) for a in f], "poisson", idx, x, w))
    prm = readout_params(gcp, max(np.abs(g).max() for _, Go in ref for g in Go))
    b = gcp.GcpBatch(clients, P, P)
    b.local_steps(1, prm, 9, 0)
    losses = b.losses()
    for i, (c, (Lo, Go)) in enumerate(zip(clients, ref)):
        assert losses[i] == pytest.approx(Lo, rel=1e-5), i
        G = recover_gradient(flat(facs[i]), flat(c.get_factors()), prm)
        o = 0
        for n, g in enumerate(Go):
            assert rel_err(G[o:o + g.size], g) <= 1e-5, (i, n, rel_err(G[o:o + g.size], g))
            o += g.size
    b.close()


def test_fedadam_rounds_match_oracle(env):
    """GCP-FedAdam (Alg. 4) on four shards of one tensor: server init, tau = 2
    local steps, reconciliation, again.  After each round every client's
    model equals the oracle's server model at 1e-5.  The oracle replays each
    round from the GPU's server model of the round before (its own moments
    carry over), as the per-step checks of the small workload do: Adam's
    normalisation turns the FP32 rounding of near-cancelling gradient entries
    into O(lr) differences of the steps, so trajectories followed
    independently drift apart over rounds while every single round agrees."""
    gcp, torch = env
    dims, R = [80, 60, 40], 8
    coords, vals = synth.uniform_sparse(dims, 6000, 77, lam=2.0)
    parts = [(coords[i::4], vals[i::4]) for i in range(4)]
    F0 = synth.factors_uniform(dims, R, 78, lo=0.1, hi=1.0)
    local = gcp.AdamParams(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, lower=0.0)
    server = gcp.AdamParams(lr=3e-2, beta1=0.6, beta2=0.99, eps=1e-8, lower=0.0)
    clients = []
    for i, (c, v) in enumerate(parts):
        ctx = gcp.gcp_create(dims, c, v, R, "poisson", seed=90 + i)
        ctx.set_factors(F0 if i == 0 else synth.factors_uniform(dims, R, 200 + i))
        clients.append(ctx)
    P = [len(v) // 2 for _, v in parts]
    b = gcp.GcpBatch(clients, P, P)
    b.server_init()
    # oracle state
    U = oracle.flat_factors(F0)
    Bs, Cs = np.zeros_like(U), np.zeros_like(U)
    Mb = [np.zeros_like(U) for _ in parts]
    Mc = [np.zeros_like(U) for _ in parts]
    it, t_local = 0, 0
    for rnd in (1, 2, 3):
        A = [U.copy() for _ in parts]
        b.local_steps(2, local, it, t_local)
        b.server_step(server, rnd)
        for i, (c, v) in enumerate(parts):
            for k in range(2):
                idx, x, w, _ = oracle.stratified_samples(90 + i, it + k, P[i], P[i], dims, c, v)
                _, G = oracle.sampled_loss_grad(dims, oracle.split_factors(A[i], dims, R), "poisson", idx, x, w)
                oracle.adam_step(A[i], Mb[i], Mc[i], np.concatenate([g.ravel() for g in G]), 1e-2, 0.9, 0.999,
                                 1e-8, 0.0, t_local + k + 1)
        oracle.fedadam_server(A, U, Bs, Cs, 3e-2, 0.6, 0.99, 1e-8, 0.0, rnd)
        it += 2
        t_local += 2
        models = [np.concatenate([a.ravel() for a in ctx.get_factors()]) for ctx in clients]
        for Ag in models:
            assert rel_err(Ag, U) <= 1e-5, (rnd, rel_err(Ag, U))
            assert np.array_equal(Ag, models[0])  # M <- U for every client
        U = models[0].astype(np.float64)  # the next round starts from the GPU's server model
    b.close()


def test_fedadam_requires_one_model_shape(env, shards):
    gcp, torch = env
    cl = make(gcp, shards[:2])
    b = gcp.GcpBatch(cl, [10, 10], [10, 10])
    with pytest.raises(gcp.GcpError):
        b.server_init()
    with pytest.raises(gcp.GcpError):
        b.server_step(gcp.AdamParams(), 1)
    b.close()


def test_batch_padded_rank_empty_client_and_unreplicated_modes(env):
    """Rank 6 (rows padded to 8 columns), a client with no samples, and a
    client whose first mode has more rows than the replica threshold: two
    local steps of the batch equal two gcp_grad + gcp_adam_step rounds of
    each client alone, and the empty client's loss is 0."""
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    specs = [([700, 40, 30], 5000, 600, 650), ([50, 60, 70], 4000, 500, 480), ([45, 35, 25], 900, 0, 0)]
    shards = []
    for i, (dims, nnz, p, q) in enumerate(specs):
        coords, vals = synth.uniform_sparse(dims, nnz, 8100 + i, lam=2.0)
        f = synth.factors_uniform(dims, 6, 8200 + i, lo=0.1, hi=1.0)
        shards.append(dict(dims=dims, coords=coords, vals=vals, factors=f, p=p, q=q, seed=8300 + i))

    def mk():
        out = []
        for s in shards:
            c = gcp.gcp_create(s["dims"], s["coords"], s["vals"], 6, "poisson", seed=s["seed"])
            c.set_factors(s["factors"])
            out.append(c)
        return out

    ref = mk()
    last = []
    for c, s in zip(ref, shards):
        for k in range(2):
            L, _ = c.grad(11 + k, s["p"], s["q"])
            c.adam_step(adam, k + 1)
        last.append(L)
    bat = mk()
    b = gcp.GcpBatch(bat, [s["p"] for s in shards], [s["q"] for s in shards])
    b.local_steps(2, adam, 11, 0)
    losses = b.losses()
    for c, r, L, Lr in zip(bat, ref, losses, last):
        A = np.concatenate([a.ravel() for a in c.get_factors()])
        Ar = np.concatenate([a.ravel() for a in r.get_factors()])
        assert rel_err(A, Ar) <= 1e-5
        assert L == pytest.approx(Lr, rel=1e-6, abs=0.0)
    assert losses[2] == 0.0
    b.close()
    for c in ref + bat:
        c.close()


@pytest.mark.parametrize("ndim,rank,tile", [(2, 8, 64), (5, 12, 16), (5, 12, 64), (4, 32, 64)])
def test_batch_orders_and_tiles_match_clients_alone(env, ndim, rank, tile):
    """Order-2, -4 and -5 client shards (the records of order 5 are 64 bytes,
    the largest staging of a 64-sample tile), padded ranks, 16 and 64
    samples per warp tile: one local step of the batch equals gcp_grad +
    gcp_adam_step on every client alone, and the batch's losses equal the
    oracle's."""
    gcp, torch = env
    adam = gcp.AdamParams(**ADAM)
    cl = synth.client_batch(5, 5100 + ndim, dim_lo=6, dim_hi=40, nnz_lo=200, nnz_hi=3000, ndim=ndim)
    sh = []
    for i, (dims, coords, vals) in enumerate(cl):
        f = synth.factors_uniform(dims, rank, 5200 + i, lo=0.1, hi=1.0)
        S = max(1, math.ceil(len(vals) / 4))
        sh.append(dict(dims=dims, coords=coords, vals=vals, factors=f, p=S, q=S + 17 * i, seed=5300 + i))

    def mk():
        out = []
        for s in sh:
            c = gcp.gcp_create(s["dims"], s["coords"], s["vals"], rank, "poisson", seed=s["seed"])
            c.set_factors(s["factors"])
            out.append(c)
        return out

    ref = mk()
    for c, s in zip(ref, sh):
        L, _ = c.grad(4, s["p"], s["q"])
        c.adam_step(adam, 1)
        s["ref_loss"] = L
    bat = mk()
    b = gcp.GcpBatch(bat, [s["p"] for s in sh], [s["q"] for s in sh])
    b.tune(samples_per_warp=tile)
    b.local_steps(1, adam, 4, 0)
    losses = b.losses()
    for c, r, s, L in zip(bat, ref, sh, losses):
        A = np.concatenate([a.ravel() for a in c.get_factors()])
        Ar = np.concatenate([a.ravel() for a in r.get_factors()])
        assert rel_err(A, Ar) <= 1e-5
        idx, x, w, _ = oracle.stratified_samples(s["seed"], 4, s["p"], s["q"], s["dims"], s["coords"], s["vals"])
        Lo, _ = oracle.sampled_loss_grad(s["dims"], s["factors"], "poisson", idx, x, w, grad=False)
        assert L == pytest.approx(Lo, rel=1e-5)
        assert L == pytest.approx(s["ref_loss"], rel=1e-6)
    b.close()
    for c in ref + bat:
        c.close()
