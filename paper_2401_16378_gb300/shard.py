"""Host side of the x-class sharding: the decomposition split over 2^k devices by the top k
bits x_hi of the XY-mask x.

Every class x of Eq. (13) is an independent 2^N-element transform (Sec. 3 remarks that the
coefficients can be evaluated independently and distributed). Device g owns the classes with
x_hi = g; with m = N - k they read only the 2^k blocks of G at block row r_hi and block column
r_hi ^ g (blocks of 2^m x 2^m). The device kernels are pauli_xhi_layout and pauli_decompose_xhi
(include/pauli.h); this module holds the index map of a shard's output, the one all-to-all that
takes a row-sharded G to the shards' block-XOR layouts, and the assembly of the shards' outputs.
None of it does arithmetic of the method.
"""
from __future__ import annotations

import numpy as np
import torch


def _spread(v: np.ndarray) -> np.ndarray:
    """Bit t of v to bit 2t."""
    v = np.asarray(v, dtype=np.uint64)
    r = np.zeros_like(v)
    for t in range(32):
        r |= ((v >> np.uint64(t)) & np.uint64(1)) << np.uint64(2 * t)
    return r


def shard_indices(N: int, k: int, x_hi: int) -> np.ndarray:
    """Pauli index n of each entry j = (z_hi << 2m) | n_lo of the shard x_hi's output
    (m = N - k): the low 2m bits of n are n_lo; qubit m + t contributes the digit of X-bit
    x_hi_t and Z-bit z_hi_t (Eq. (2): even bit x ^ z, odd bit z)."""
    if not 0 <= k < N or not 0 <= x_hi < (1 << k):
        raise ValueError("need 0 <= k < N and 0 <= x_hi < 2^k")
    m = N - k
    j = np.arange((4 ** N) >> k, dtype=np.uint64)
    n_lo = j & np.uint64((1 << (2 * m)) - 1)
    z_hi = j >> np.uint64(2 * m)
    top = _spread(np.uint64(x_hi) ^ z_hi) | (_spread(z_hi) << np.uint64(1))
    return n_lo | (top << np.uint64(2 * m))


def block_xor_from_rows(G_rows: torch.Tensor, N: int, k: int, group=None) -> torch.Tensor:
    """All-to-all redistribution of a row-sharded G into this rank's block-XOR layout.

    2^k ranks; rank w holds G_rows = G[w M : (w + 1) M, :] (M = 2^(N - k) rows of 2^N elements)
    and owns the shard x_hi = w. Rank w sends to rank g its column block w ^ g (an M x M block,
    the block (w, w ^ g) that shard g needs); the chunks arrive in rank order, so the received
    buffer is rank g's layout L (D rows of M elements, blocks stacked by r_hi). Returns L with
    shape (2^N, M) on G_rows' device."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if world != 1 << k:
        raise ValueError(f"world size {world} is not 2^k = {1 << k}")
    M = 1 << (N - k)
    if tuple(G_rows.shape) != (M, 1 << N):
        raise ValueError(f"G_rows must have shape ({M}, {1 << N})")
    blocks = G_rows.reshape(M, world, M)  # [row][column block][column]
    send = torch.stack([blocks[:, rank ^ g, :] for g in range(world)]).contiguous()  # [dest g][row][col]
    recv = torch.empty_like(send)
    # exchanged as real pairs: collective backends need not support complex tensors
    dist.all_to_all_single(torch.view_as_real(recv), torch.view_as_real(send), group=group)
    return recv.reshape(1 << N, M)


def assemble(shard_outputs, N: int, k: int) -> np.ndarray:
    """The full coefficient vector from the 2^k shards' outputs (host arrays, in x_hi order)."""
    outs = [np.asarray(o) for o in shard_outputs]
    if len(outs) != 1 << k:
        raise ValueError("need one output per shard")
    full = np.empty(4 ** N, dtype=outs[0].dtype)
    seen = np.zeros(4 ** N, dtype=bool)
    for g, o in enumerate(outs):
        idx = shard_indices(N, k, g).astype(np.int64)
        if o.size != idx.size:
            raise ValueError(f"shard {g} holds {o.size} values, expected {idx.size}")
        full[idx] = o
        seen[idx] = True
    if not seen.all():
        raise AssertionError("the shards do not cover every coefficient")
    return full
