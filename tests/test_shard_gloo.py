"""Chain sharding over ranks, on CPU processes with the gloo backend.

Each rank runs its contiguous chain range (global chain ids through
chain_offset) and rank 0 gathers state and moments in rank order; the result
must equal one run over all chains bit for bit, for the three Gibbs models and
for a ragged split.  The per-rank work here is the oracle, standing in for a
GPU rank (the device path is shown equal to the oracle by the GPU parity
tests, and its chain_offset sharding by the split-call tests there).
"""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1412_4825_gb300 import inputs, shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

SEED = 0x5EED5
PRIOR = (2.0, 1.0, 0.0, 0.01)


def test_chain_range_partitions():
    for n in (0, 1, 7, 1000, 65536, 65537):
        for world in (1, 2, 3, 8):
            ranges = [shard.chain_range(n, world, r) for r in range(world)]
            assert ranges[0][0] == 0
            for (o0, c0), (o1, _) in zip(ranges, ranges[1:]):
                assert o0 + c0 == o1
            assert sum(c for _, c in ranges) == n
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1
    assert shard.weak_range(65536, 3) == (3 * 65536, 65536)
    with pytest.raises(ValueError):
        shard.chain_range(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_tri, n_ng, n_lda, sweeps):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nobs, xbar, sc = inputs.normal_gamma_data(n_ng, seed=7)
        alpha, _, _ = inputs.lda_alpha(n_lda, K=16, seed=8)
        t_max = shard.max_over_ranks(dist, 1.0 + rank)
        assert t_max == float(world)

        # triangle (Eq. 1)
        off, cnt = shard.chain_range(n_tri, world, rank)
        r = O.gibbs_triangle(SEED, cnt, sweeps, chain_offset=off)
        xy = shard.gather_rows(dist, torch.from_numpy(r["xy"]), n_tri, world, rank)
        mom = shard.gather_rows(dist, torch.from_numpy(r["mom"]), n_tri, world, rank)
        if rank == 0:
            ref = O.gibbs_triangle(SEED, n_tri, sweeps)
            assert np.array_equal(xy.numpy().view(np.uint64), ref["xy"].view(np.uint64))
            assert np.array_equal(mom.numpy().view(np.uint64), ref["mom"].view(np.uint64))

        # normal-gamma: a rank's data rows are its slice of the global data
        off, cnt = shard.chain_range(n_ng, world, rank)
        sl = slice(off, off + cnt)
        r = O.gibbs_normal_gamma(SEED, sweeps, nobs[sl], xbar[sl], sc[sl], prior=PRIOR, chain_offset=off)
        st = shard.gather_rows(dist, torch.from_numpy(r["state"]), n_ng, world, rank)
        pos = shard.gather_rows(dist, torch.from_numpy(r["pos"].view(np.int64)), n_ng, world, rank)
        mom = shard.gather_rows(dist, torch.from_numpy(r["mom"]), n_ng, world, rank)
        if rank == 0:
            ref = O.gibbs_normal_gamma(SEED, sweeps, nobs, xbar, sc, prior=PRIOR)
            assert np.array_equal(st.numpy().view(np.uint64), ref["state"].view(np.uint64))
            assert np.array_equal(pos.numpy().view(np.uint64), ref["pos"])
            assert np.array_equal(mom.numpy().view(np.uint64), ref["mom"].view(np.uint64))

        # LDA document-topic step
        off, cnt = shard.chain_range(n_lda, world, rank)
        r = O.gibbs_lda(SEED, sweeps, alpha[off:off + cnt], doc_offset=off)
        th = shard.gather_rows(dist, torch.from_numpy(r["theta"]), n_lda, world, rank)
        mom = shard.gather_rows(dist, torch.from_numpy(r["mom"]), n_lda, world, rank)
        if rank == 0:
            ref = O.gibbs_lda(SEED, sweeps, alpha)
            assert np.array_equal(th.numpy().view(np.uint64), ref["theta"].view(np.uint64))
            assert np.array_equal(mom.numpy().view(np.uint64), ref["mom"].view(np.uint64))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_sharded_equals_whole_gloo(world):
    O.lib()  # build the oracle before the ranks start
    mp.start_processes(_rank_main, args=(world, _free_port(), 257, 301, 37, 40), nprocs=world,
                       join=True, start_method="spawn")


def _lda_rank_main(rank, world, port, n_docs, sweeps, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        corpus = inputs.lda_corpus(n_docs, K=16, V=200, len_lo=5, len_hi=80, seed=21)
        full = inputs.lda_initial_state(corpus, seed=22)
        off, cnt = shard.chain_range(n_docs, world, rank)
        sub = dict(K=corpus["K"], V=corpus["V"], doc_ptr=corpus["doc_ptr"][off:off + cnt + 1], words=corpus["words"])
        st = {k: v.copy() for k, v in full.items()}
        st["ndk"] = np.ascontiguousarray(full["ndk"][off:off + cnt])
        st["zpos"] = np.ascontiguousarray(full["zpos"][off:off + cnt])
        K, V = corpus["K"], corpus["V"]
        for _ in range(sweeps):
            dnkw, dnk = O.lda_z_sweep(SEED, sub, st, 0.1, 0.01, doc_offset=off)
            d = torch.from_numpy(np.concatenate([dnkw.ravel(), dnk]))
            shard.lda_exchange(dist, d)
            st["nkw"] += d[: V * K].numpy().reshape(V, K)
            st["nk"] += d[V * K:].numpy()
        t0, t1 = int(corpus["doc_ptr"][off]), int(corpus["doc_ptr"][off + cnt])
        ndk = shard.gather_rows(dist, torch.from_numpy(st["ndk"]), n_docs, world, rank)
        z = torch.from_numpy(st["z"][t0:t1].astype(np.int32))
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([t1 - t0]))
        width = int(max(x.item() for x in sizes))
        pad = torch.zeros(width, dtype=torch.int32)
        pad[: t1 - t0] = z
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        if rank == 0:
            zall = torch.cat([p[: int(c.item())] for p, c in zip(parts, sizes)]).numpy()
            out_q.put((ndk.numpy(), zall, st["nkw"], st["nk"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_lda_full_sharded_exchange_equals_one_run(world):
    """The full LDA step on `world` gloo ranks -- documents split by
    chain_range, each sweep's count changes summed over the ranks with
    lda_exchange -- gives the single run's topics and counts exactly."""
    n_docs, sweeps = 37, 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    mp.start_processes(_lda_rank_main, args=(world, port, n_docs, sweeps, q), nprocs=world, join=True,
                       start_method="spawn")
    ndk, z, nkw, nk = q.get(timeout=60)
    corpus = inputs.lda_corpus(n_docs, K=16, V=200, len_lo=5, len_hi=80, seed=21)
    ref = inputs.lda_initial_state(corpus, seed=22)
    O.lda_full(SEED, sweeps, corpus, ref, alpha=0.1, beta=0.01, theta_draws=False)
    assert np.array_equal(ndk, ref["ndk"]) and np.array_equal(z, ref["z"].astype(np.int32))
    assert np.array_equal(nkw, ref["nkw"]) and np.array_equal(nk, ref["nk"])
