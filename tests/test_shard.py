"""x-class sharding, host side (no GPU): the index map of a shard's output, the block split of
Eq. (13) the shard kernel relies on (checked against the oracle), and the all-to-all that takes
a row-sharded G to the shards' block-XOR layouts, run as gloo ranks (world size 2 and 4)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_16378_gb300 import shard, workloads  # noqa: E402


def _x_mask(n: np.ndarray, N: int) -> np.ndarray:
    """XY-mask of Pauli indices, digit by digit (digit 1 = X, 2 = Y: x_t set)."""
    x = np.zeros_like(n)
    for t in range(N):
        d = (n >> np.uint64(2 * t)) & np.uint64(3)
        x |= ((d == 1) | (d == 2)).astype(np.uint64) << np.uint64(t)
    return x


def _layout(G: np.ndarray, k: int, g: int) -> np.ndarray:
    """Block-XOR layout of shard g, element by element from its definition."""
    D = G.shape[0]
    m = D.bit_length() - 1 - k
    M = 1 << m
    L = np.empty((D, M), dtype=G.dtype)
    for r in range(D):
        cb = (r >> m) ^ g
        L[r] = G[r, cb * M:(cb + 1) * M]
    return L


@pytest.mark.parametrize("N,k", [(3, 1), (4, 2), (5, 1), (5, 3), (6, 5)])
def test_shard_indices_partition_the_coefficients(N, k):
    seen = np.zeros(4 ** N, dtype=np.int64)
    for g in range(1 << k):
        n = shard.shard_indices(N, k, g)
        assert n.size == (4 ** N) >> k
        assert np.all((_x_mask(n, N) >> np.uint64(N - k)) == g), "every entry's top X bits are x_hi"
        seen[n.astype(np.int64)] += 1
    assert np.all(seen == 1)


def test_shard_indices_low_bits_are_the_block_index():
    N, k = 5, 2
    m = N - k
    for g in range(4):
        n = shard.shard_indices(N, k, g)
        j = np.arange(n.size, dtype=np.uint64)
        assert np.all((n & np.uint64(4 ** m - 1)) == (j & np.uint64(4 ** m - 1)))


@pytest.mark.parametrize("N,k", [(4, 1), (5, 2), (6, 3)])
def test_block_split_of_the_sum_matches_the_oracle(N, k):
    """c(x, z) = 2^-k i^popc(x_hi & z_hi) sum_{r_hi} (-1)^popc(r_hi & z_hi) c_B(r_hi)(x_lo, z_lo),
    with c_B from the oracle on each m-qubit block, against the oracle on the full matrix."""
    G = workloads.gaussian_complex(N, 40 + N)
    m, M = N - k, 1 << (N - k)
    want = oracle.decompose_full(G)
    for g in range(1 << k):
        L = _layout(G, k, g)
        blocks = [oracle.decompose_full(L[rh * M:(rh + 1) * M]) for rh in range(1 << k)]
        n = shard.shard_indices(N, k, g)
        got = np.empty(n.size, dtype=np.complex128)
        for zh in range(1 << k):
            acc = np.zeros(4 ** m, dtype=np.complex128)
            for rh in range(1 << k):
                acc += (-1) ** bin(rh & zh).count("1") * blocks[rh]
            got[zh * 4 ** m:(zh + 1) * 4 ** m] = acc * 1j ** bin(g & zh).count("1") / (1 << k)
        np.testing.assert_allclose(got, want[n.astype(np.int64)], rtol=0, atol=1e-13 * np.max(np.abs(G)))


def test_assemble_rejects_missing_and_misshaped_shards():
    N, k = 3, 1
    outs = [np.zeros((4 ** N) >> k, dtype=np.complex128) for _ in range(2)]
    assert shard.assemble(outs, N, k).shape == (4 ** N,)
    with pytest.raises(ValueError):
        shard.assemble(outs[:1], N, k)
    with pytest.raises(ValueError):
        shard.assemble([outs[0], outs[1][:-1]], N, k)
    with pytest.raises(ValueError):
        shard.shard_indices(N, N, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, N, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle as orc
    from paper_2401_16378_gb300 import shard as sh
    from paper_2401_16378_gb300 import workloads as wl

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        k = world.bit_length() - 1
        M = 1 << (N - k)
        G = wl.gaussian_complex(N, 90 + N)  # every rank draws the same matrix, then keeps its rows
        rows = torch.from_numpy(G[rank * M:(rank + 1) * M].copy())
        L = sh.block_xor_from_rows(rows, N, k).numpy()
        layout_ok = bool(np.array_equal(L, _layout(G, k, rank)))
        # this rank's coefficients from its own blocks only: the other blocks of G stay zero
        Gs = np.zeros_like(G)
        for rh in range(world):
            cb = rh ^ rank
            Gs[rh * M:(rh + 1) * M, cb * M:(cb + 1) * M] = L[rh * M:(rh + 1) * M]
        mine = orc.decompose_at(Gs, sh.shard_indices(N, k, rank))
        parts = [torch.empty(mine.size, dtype=torch.complex128) for _ in range(world)]
        dist.all_gather([torch.view_as_real(p) for p in parts], torch.view_as_real(torch.from_numpy(mine)))
        ok = None
        if rank == 0:
            full = sh.assemble([p.numpy() for p in parts], N, k)
            ok = float(np.max(np.abs(full - orc.decompose_full(G))) / np.max(np.abs(G)))
        q.put((rank, layout_ok, ok))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,N", [(2, 5), (4, 6)])
def test_row_sharded_matrix_reaches_the_shards_over_gloo(world, N):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, N, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted((q.get(timeout=10) for _ in range(world)), key=lambda t: t[0])
    assert all(layout_ok for _, layout_ok, _ in got), "each rank received its block-XOR layout"
    assert got[0][2] < 1e-14, "the union of the shards is every coefficient of the oracle"
