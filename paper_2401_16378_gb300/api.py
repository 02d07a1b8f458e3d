"""Python binding of libpauli: the C entry points under the same names, taking torch tensors.

Argument marshalling only -- every step of the computation runs in libpauli's CUDA kernels.
PyTorch provides device memory and the current stream.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import _lib
from ._lib import PAULI_AUTO, PAULI_C64, PAULI_C128, PAULI_PLAIN, PAULI_XORDIAG, PauliError, check  # noqa: F401

_METHODS = {"auto": PAULI_AUTO, "plain": PAULI_PLAIN, "xordiag": PAULI_XORDIAG}
_DTYPES = {torch.complex64: PAULI_C64, torch.complex128: PAULI_C128}


def _method(m) -> int:
    if isinstance(m, str):
        return _METHODS[m]
    return int(m)


def _dtype(t: torch.Tensor) -> int:
    try:
        return _DTYPES[t.dtype]
    except KeyError:
        raise TypeError(f"dtype {t.dtype} is not complex64 or complex128") from None


def _stream(stream) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _qubits_of_matrix(G: torch.Tensor) -> int:
    if G.dim() < 2 or G.shape[-1] != G.shape[-2]:
        raise ValueError("G must have shape (..., D, D)")
    D = G.shape[-1]
    if D < 2 or D & (D - 1):
        raise ValueError("D must be a power of two >= 2")
    return D.bit_length() - 1


def _qubits_of_coeffs(c: torch.Tensor) -> int:
    n = c.shape[-1]
    N = (n.bit_length() - 1) // 2
    if n < 4 or 4 ** N != n:
        raise ValueError("the last dimension of c must be 4^N")
    return N


def _device_tensor(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def pauli_decompose(G: torch.Tensor, out: torch.Tensor | None = None, method="auto", stream=None) -> torch.Tensor:
    """c_n = 2^-N Tr(P_n G) for a (..., 2^N, 2^N) complex CUDA tensor; returns (..., 4^N)."""
    _device_tensor(G, "G")
    N = _qubits_of_matrix(G)
    count = G.numel() // (4 ** N)
    if out is None:
        out = torch.empty(G.shape[:-2] + (4 ** N,), dtype=G.dtype, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != G.dtype or out.numel() != G.numel():
        raise ValueError("out must match G in dtype and number of elements")
    check(_lib.load().pauli_decompose(G.data_ptr(), N, count, _dtype(G), out.data_ptr(), _method(method),
                                      _stream(stream)))
    return out


def pauli_decompose_workspace_size(N: int, count: int = 1, dtype: torch.dtype = torch.complex128,
                                   method="auto") -> int:
    """Bytes of caller scratch that pauli_decompose_ws needs (0 when it needs none)."""
    n = ctypes.c_size_t(0)
    check(_lib.load().pauli_decompose_workspace_size(int(N), int(count), _DTYPES[dtype], _method(method),
                                                     ctypes.byref(n)))
    return int(n.value)


def pauli_decompose_ws(G: torch.Tensor, workspace: torch.Tensor | None, out: torch.Tensor | None = None,
                       method="auto", stream=None) -> torch.Tensor:
    """pauli_decompose with caller-provided scratch (a CUDA tensor of at least
    pauli_decompose_workspace_size bytes); the library allocates nothing."""
    _device_tensor(G, "G")
    N = _qubits_of_matrix(G)
    count = G.numel() // (4 ** N)
    if out is None:
        out = torch.empty(G.shape[:-2] + (4 ** N,), dtype=G.dtype, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != G.dtype or out.numel() != G.numel():
        raise ValueError("out must match G in dtype and number of elements")
    wp, wb = 0, 0
    if workspace is not None:
        _device_tensor(workspace, "workspace")
        wp, wb = workspace.data_ptr(), workspace.numel() * workspace.element_size()
    check(_lib.load().pauli_decompose_ws(G.data_ptr(), N, count, _dtype(G), out.data_ptr(), _method(method),
                                         ctypes.c_void_p(wp), wb, _stream(stream)))
    return out


def workspace_status(workspace: torch.Tensor, stream=None) -> None:
    """Synchronise the stream and raise PauliError if the last pauli_decompose_ws call that used
    `workspace` timed out in a bounded device wait."""
    check(_lib.load().pauli_workspace_status(ctypes.c_void_p(workspace.data_ptr()), _stream(stream)))


def release_workspaces(stream=None) -> None:
    """Free the library-owned scratch of the current device for `stream` (after synchronising it)."""
    check(_lib.load().pauli_release_workspaces(_stream(stream)))


def pauli_decompose_hermitian(G: torch.Tensor, out: torch.Tensor | None = None, method="auto", stream=None,
                              upper: bool = False) -> torch.Tensor:
    """Re c_n for a (..., 2^N, 2^N) complex CUDA tensor (all of c_n when G is Hermitian); returns
    a real (..., 4^N) tensor of G's precision. upper=True: G is Hermitian and only its upper
    triangle (and the diagonal's real parts) is read -- half the bytes (N <= 14)."""
    _device_tensor(G, "G")
    N = _qubits_of_matrix(G)
    count = G.numel() // (4 ** N)
    rdt = {torch.complex64: torch.float32, torch.complex128: torch.float64}.get(G.dtype)
    if rdt is None:
        raise TypeError(f"dtype {G.dtype} is not complex64 or complex128")
    if out is None:
        out = torch.empty(G.shape[:-2] + (4 ** N,), dtype=rdt, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != rdt or out.numel() != G.numel():
        raise ValueError("out must hold one real of G's precision per coefficient")
    fn = _lib.load().pauli_decompose_hermitian_upper if upper else _lib.load().pauli_decompose_hermitian
    check(fn(G.data_ptr(), N, count, _dtype(G), out.data_ptr(), _method(method), _stream(stream)))
    return out


def pauli_decompose_real(G: torch.Tensor, out: torch.Tensor | None = None, method="auto", stream=None) -> torch.Tensor:
    """For a real float64 (..., 2^N, 2^N) CUDA tensor: the real a_n with c_n = i^(k mod 2) a_n
    (k = number of Y factors of P_n), a float64 (..., 4^N) tensor."""
    _device_tensor(G, "G")
    if G.dtype != torch.float64:
        raise TypeError("G must be float64")
    N = _qubits_of_matrix(G)
    if out is None:
        out = torch.empty(G.shape[:-2] + (4 ** N,), dtype=torch.float64, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != torch.float64 or out.numel() != G.numel():
        raise ValueError("out must hold one float64 per coefficient")
    check(_lib.load().pauli_decompose_real(G.data_ptr(), N, G.numel() // 4 ** N, PAULI_C128, out.data_ptr(),
                                           _method(method), _stream(stream)))
    return out


def pauli_compose(c: torch.Tensor, out: torch.Tensor | None = None, scale_exp: int = 0, stream=None) -> torch.Tensor:
    """G = 2^scale_exp sum_n c_n P_n for a (..., 4^N) complex CUDA tensor; returns (..., 2^N, 2^N)."""
    _device_tensor(c, "c")
    N = _qubits_of_coeffs(c)
    count = c.numel() // (4 ** N)
    if out is None:
        out = torch.empty(c.shape[:-1] + (1 << N, 1 << N), dtype=c.dtype, device=c.device)
    _device_tensor(out, "out")
    if out.dtype != c.dtype or out.numel() != c.numel():
        raise ValueError("out must match c in dtype and number of elements")
    check(_lib.load().pauli_compose(c.data_ptr(), N, count, _dtype(c), out.data_ptr(), int(scale_exp),
                                    _stream(stream)))
    return out


_REAL = {torch.complex64: torch.float32, torch.complex128: torch.float64}


def _weights(c: torch.Tensor, w: torch.Tensor, N: int) -> torch.Tensor:
    _device_tensor(w, "w")
    if w.dtype != _REAL[c.dtype] or w.numel() != 4 ** N:
        raise ValueError(f"w must hold 4^N values of {_REAL[c.dtype]}")
    return w


def pauli_weighted_norm(c: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """sum over the batch and n of w_n |c_n|^2 for a (..., 4^N) CUDA tensor; a 0-dim real tensor."""
    _device_tensor(c, "c")
    N = _qubits_of_coeffs(c)
    _weights(c, w, N)
    if out is None:
        out = torch.empty((), dtype=_REAL[c.dtype], device=c.device)
    _device_tensor(out, "out")
    if out.dtype != _REAL[c.dtype] or out.numel() != 1:
        raise ValueError("out must be one real of c's precision")
    check(_lib.load().pauli_weighted_norm(c.data_ptr(), N, c.numel() // 4 ** N, _dtype(c), w.data_ptr(),
                                          out.data_ptr(), _stream(stream)))
    return out


def pauli_weighted_norm_grad(c: torch.Tensor, w: torch.Tensor, g: torch.Tensor | None = None,
                             out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """2 g w_n c_n (g a one-element real CUDA tensor, or None for 1); out may be c itself."""
    _device_tensor(c, "c")
    N = _qubits_of_coeffs(c)
    _weights(c, w, N)
    gp = None
    if g is not None:
        _device_tensor(g, "g")
        if g.dtype != _REAL[c.dtype] or g.numel() != 1:
            raise ValueError("g must be one real of c's precision")
        gp = g.data_ptr()
    if out is None:
        out = torch.empty_like(c)
    _device_tensor(out, "out")
    if out.dtype != c.dtype or out.numel() != c.numel():
        raise ValueError("out must match c in dtype and number of elements")
    check(_lib.load().pauli_weighted_norm_grad(c.data_ptr(), N, c.numel() // 4 ** N, _dtype(c), w.data_ptr(), gp,
                                               out.data_ptr(), _stream(stream)))
    return out


def pauli_decompose_weighted_norm(G: torch.Tensor, w: torch.Tensor, out: torch.Tensor | None = None,
                                  loss: torch.Tensor | None = None, method="auto", stream=None):
    """(c, L): the decomposition of G and L = sum over the batch and n of w_n |c_n|^2, computed
    together (one fused kernel for N 6..12)."""
    _device_tensor(G, "G")
    N = _qubits_of_matrix(G)
    count = G.numel() // (4 ** N)
    if out is None:
        out = torch.empty(G.shape[:-2] + (4 ** N,), dtype=G.dtype, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != G.dtype or out.numel() != G.numel():
        raise ValueError("out must match G in dtype and number of elements")
    _weights(G, w, N)
    if loss is None:
        loss = torch.empty((), dtype=_REAL[G.dtype], device=G.device)
    _device_tensor(loss, "loss")
    if loss.dtype != _REAL[G.dtype] or loss.numel() != 1:
        raise ValueError("loss must be one real of G's precision")
    check(_lib.load().pauli_decompose_weighted_norm(G.data_ptr(), N, count, _dtype(G), out.data_ptr(), w.data_ptr(),
                                                    loss.data_ptr(), _method(method), _stream(stream)))
    return out, loss


def pauli_compose_weighted(c: torch.Tensor, w: torch.Tensor, g: torch.Tensor | None = None,
                           out: torch.Tensor | None = None, scale_exp: int = 0, stream=None) -> torch.Tensor:
    """G = 2^scale_exp sum_n g w_n c_n P_n for a (..., 4^N) CUDA tensor, N <= 12 (g: one real, or None)."""
    _device_tensor(c, "c")
    N = _qubits_of_coeffs(c)
    count = c.numel() // (4 ** N)
    _weights(c, w, N)
    gp = None
    if g is not None:
        _device_tensor(g, "g")
        if g.dtype != _REAL[c.dtype] or g.numel() != 1:
            raise ValueError("g must be one real of c's precision")
        gp = g.data_ptr()
    if out is None:
        out = torch.empty(c.shape[:-1] + (1 << N, 1 << N), dtype=c.dtype, device=c.device)
    _device_tensor(out, "out")
    if out.dtype != c.dtype or out.numel() != c.numel():
        raise ValueError("out must match c in dtype and number of elements")
    check(_lib.load().pauli_compose_weighted(c.data_ptr(), N, count, _dtype(c), w.data_ptr(), gp, out.data_ptr(),
                                             int(scale_exp), _stream(stream)))
    return out


def pauli_coeffs_at(G: torch.Tensor, idx: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """c_n for the listed n (a CUDA int64/uint64 tensor), O(2^N) each, no scratch memory."""
    _device_tensor(G, "G")
    _device_tensor(idx, "idx")
    if idx.dtype not in (torch.int64, torch.uint64):
        raise TypeError("idx must be int64 or uint64")
    N = _qubits_of_matrix(G)
    if G.dim() != 2:
        raise ValueError("pauli_coeffs_at takes one matrix")
    k = idx.numel()
    if out is None:
        out = torch.empty(k, dtype=G.dtype, device=G.device)
    _device_tensor(out, "out")
    check(_lib.load().pauli_coeffs_at(G.data_ptr(), N, _dtype(G), idx.data_ptr(), k, out.data_ptr(), _stream(stream)))
    return out


def _ptr_array(ptrs: Sequence[int]):
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def pauli_decompose_list(Gs: Sequence[torch.Tensor], outs: Sequence[torch.Tensor] | None = None, method="auto",
                         stream=None) -> list[torch.Tensor]:
    """One launch per matrix (matrices of different N); returns the list of coefficient tensors."""
    if not Gs:
        return []
    dt = _dtype(Gs[0])
    Ns = [_qubits_of_matrix(_device_tensor(G, "G")) for G in Gs]
    if outs is None:
        outs = [torch.empty(4 ** N, dtype=G.dtype, device=G.device) for G, N in zip(Gs, Ns)]
    gp, keep1 = _ptr_array([G.data_ptr() for G in Gs])
    op, keep2 = _ptr_array([o.data_ptr() for o in outs])
    narr = (ctypes.c_int * len(Ns))(*Ns)
    check(_lib.load().pauli_decompose_list(gp, narr, len(Gs), dt, op, _method(method), _stream(stream)))
    return list(outs)


def pauli_xhi_layout(G: torch.Tensor, k: int, x_hi: int, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """Block-XOR layout of the x-class shard x_hi of a (2^N, 2^N) CUDA matrix: a (2^N, 2^(N-k))
    tensor, row r holding G[r, ((r >> (N-k)) ^ x_hi) << (N-k) | j] at column j."""
    _device_tensor(G, "G")
    N = _qubits_of_matrix(G)
    if G.dim() != 2:
        raise ValueError("G must be one (2^N, 2^N) matrix")
    if out is None:
        out = torch.empty((1 << N, 1 << (N - k)) if 0 <= k < N else (0,), dtype=G.dtype, device=G.device)
    _device_tensor(out, "out")
    if out.dtype != G.dtype or out.numel() != G.numel() >> k:
        raise ValueError("out must match G in dtype and hold 4^N / 2^k elements")
    check(_lib.load().pauli_xhi_layout(G.data_ptr(), N, int(k), int(x_hi), _dtype(G), out.data_ptr(),
                                       _stream(stream)))
    return out


def pauli_decompose_xhi(L: torch.Tensor, N: int, k: int, x_hi: int, out: torch.Tensor | None = None,
                        method="auto", stream=None) -> torch.Tensor:
    """Coefficients of the x-class shard x_hi from its block-XOR layout L (4^N / 2^k elements):
    out[(z_hi << 2(N-k)) | n_lo] = c_n for the n with top XY-mask bits x_hi (shard_indices)."""
    _device_tensor(L, "L")
    if out is None:
        out = torch.empty(L.numel(), dtype=L.dtype, device=L.device)
    _device_tensor(out, "out")
    if out.dtype != L.dtype or out.numel() != L.numel():
        raise ValueError("out must match L in dtype and number of elements")
    if 0 <= k < N and L.numel() != (4 ** N) >> k:
        raise ValueError("L must hold 4^N / 2^k elements")
    check(_lib.load().pauli_decompose_xhi(L.data_ptr(), int(N), int(k), int(x_hi), _dtype(L), out.data_ptr(),
                                          _method(method), _stream(stream)))
    return out


def pauli_compose_batched(cs: Sequence[torch.Tensor], outs: Sequence[torch.Tensor] | None = None, scale_exp: int = 0,
                          stream=None) -> list[torch.Tensor]:
    """G_b = 2^scale_exp sum_n c_b[n] P_n for coefficient vectors of different N, in one launch."""
    if not cs:
        return []
    dt = _dtype(cs[0])
    Ns = [_qubits_of_coeffs(_device_tensor(c, "c")) for c in cs]
    if outs is None:
        outs = [torch.empty((1 << N, 1 << N), dtype=c.dtype, device=c.device) for c, N in zip(cs, Ns)]
    cp, keep1 = _ptr_array([c.data_ptr() for c in cs])
    op, keep2 = _ptr_array([o.data_ptr() for o in outs])
    narr = (ctypes.c_int * len(Ns))(*Ns)
    check(_lib.load().pauli_compose_batched(cp, narr, len(cs), dt, op, int(scale_exp), _stream(stream)))
    return list(outs)


def pauli_decompose_host(G_host: torch.Tensor, out_host: torch.Tensor, G_dev: torch.Tensor, out_dev: torch.Tensor,
                         method="auto", stream=None) -> None:
    """Host -> device copy, decomposition and device -> host copy on one stream (asynchronous;
    pinned host tensors make the copies asynchronous). Synchronise the stream before reading
    out_host."""
    for t, name in ((G_host, "G_host"), (out_host, "out_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    _device_tensor(G_dev, "G_dev")
    _device_tensor(out_dev, "out_dev")
    N = _qubits_of_matrix(G_host)
    count = G_host.numel() // (4 ** N)
    for t in (out_host, G_dev, out_dev):
        if t.numel() != G_host.numel() or t.dtype != G_host.dtype:
            raise ValueError("all four buffers must hold the same number of elements of one dtype")
    check(_lib.load().pauli_decompose_host(G_host.data_ptr(), N, count, _dtype(G_host), out_host.data_ptr(),
                                           G_dev.data_ptr(), out_dev.data_ptr(), _method(method), _stream(stream)))


def pauli_decompose_host_stream(G_hosts: Sequence[torch.Tensor], out_hosts: Sequence[torch.Tensor],
                                G_devs: Sequence[torch.Tensor], out_devs: Sequence[torch.Tensor], method="auto",
                                stream=None) -> None:
    """Decompose a list of host matrices of one N: copy-in, decomposition and copy-out pipelined
    over the library's streams and the two device buffer pairs G_devs[0..1], out_devs[0..1]
    (asynchronous; pinned host tensors; synchronise `stream` before reading out_hosts)."""
    if len(G_hosts) != len(out_hosts) or not G_hosts:
        raise ValueError("one output per input matrix, at least one")
    if len(G_devs) != 2 or len(out_devs) != 2:
        raise ValueError("two device input buffers and two device output buffers")
    N = _qubits_of_matrix(G_hosts[0])
    for t in list(G_hosts) + list(out_hosts):
        if t.is_cuda or not t.is_contiguous() or t.numel() != 4 ** N or t.dtype != G_hosts[0].dtype:
            raise ValueError("host buffers: contiguous, on the host, 4^N elements of one complex dtype")
    for t in list(G_devs) + list(out_devs):
        _device_tensor(t, "device buffer")
        if t.numel() != 4 ** N or t.dtype != G_hosts[0].dtype:
            raise ValueError("device buffers: 4^N elements of the host buffers' dtype")
    gh, k1 = _ptr_array([t.data_ptr() for t in G_hosts])
    oh, k2 = _ptr_array([t.data_ptr() for t in out_hosts])
    gd, k3 = _ptr_array([t.data_ptr() for t in G_devs])
    od, k4 = _ptr_array([t.data_ptr() for t in out_devs])
    check(_lib.load().pauli_decompose_host_stream(gh, oh, len(G_hosts), N, _dtype(G_hosts[0]), gd, od, _method(method),
                                                  _stream(stream)))


class PauliPlan:
    """One persistent launch decomposing a batch of matrices of uneven N (pauli_plan_*)."""

    def __init__(self, Ns: Sequence[int], dtype: torch.dtype = torch.complex128, threads_per_block: int = 0,
                 blocks_per_sm: int = 0, hermitian: bool = False):
        """hermitian=True: the matrices are Hermitian, read from their upper triangle; outputs
        are real tensors of 4^N values (pauli_plan_create_hermitian)."""
        self._lib = _lib.load()
        self.Ns = [int(n) for n in Ns]
        self.dtype = dtype
        self.hermitian = bool(hermitian)
        if not threads_per_block:  # the autotuned CTA size on this GPU model, if measured
            from . import autotune

            threads_per_block = autotune.plan_threads(dtype)
        narr = (ctypes.c_int * len(self.Ns))(*self.Ns)
        h = ctypes.c_void_p()
        create = self._lib.pauli_plan_create_hermitian if self.hermitian else self._lib.pauli_plan_create
        check(create(narr, len(self.Ns), _DTYPES[dtype], int(threads_per_block), int(blocks_per_sm), ctypes.byref(h)))
        self._h = h
        self._bound = None

    def bind(self, Gs: Sequence[torch.Tensor], outs: Sequence[torch.Tensor]) -> None:
        if len(Gs) != len(self.Ns) or len(outs) != len(self.Ns):
            raise ValueError("one input and one output per planned matrix")
        gp, k1 = _ptr_array([_device_tensor(G, "G").data_ptr() for G in Gs])
        op, k2 = _ptr_array([_device_tensor(o, "out").data_ptr() for o in outs])
        check(self._lib.pauli_plan_bind(self._h, gp, op))
        self._bound = (list(Gs), list(outs))  # keep the tensors alive while bound

    def execute(self, stream=None) -> None:
        check(self._lib.pauli_plan_execute(self._h, _stream(stream)))

    def graph_launch(self, stream=None) -> None:
        check(self._lib.pauli_plan_graph_launch(self._h, _stream(stream)))

    def status(self) -> int:
        """Synchronise and return the plan's status (0 = PAULI_OK, 8 = PAULI_ERR_TIMEOUT)."""
        return int(self._lib.pauli_plan_status(self._h))

    def set_stall(self, stall: bool) -> None:
        check(self._lib.pauli_plan_set_stall(self._h, int(bool(stall))))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.pauli_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PauliDecompose(torch.autograd.Function):
    """c = decompose(G) with the hand-written adjoint: grad_G = 2^-N compose(grad_c)."""

    @staticmethod
    def forward(ctx, G: torch.Tensor, method="auto"):
        ctx.N = _qubits_of_matrix(G)
        return pauli_decompose(G.contiguous(), method=method)

    @staticmethod
    def backward(ctx, grad_c: torch.Tensor):
        return pauli_compose(grad_c.contiguous(), scale_exp=-ctx.N), None


def decompose_autograd(G: torch.Tensor, method="auto") -> torch.Tensor:
    return PauliDecompose.apply(G, method)


class PauliWeightedNorm(torch.autograd.Function):
    """L = sum w_n |c_n|^2 over the batch, with the hand-written gradient 2 g w c (w is constant)."""

    @staticmethod
    def forward(ctx, c: torch.Tensor, w: torch.Tensor):
        c = c.contiguous()
        ctx.save_for_backward(c, w)
        return pauli_weighted_norm(c, w)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        c, w = ctx.saved_tensors
        return pauli_weighted_norm_grad(c, w, g.contiguous()), None


def weighted_norm_autograd(c: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    return PauliWeightedNorm.apply(c, w)


class PauliDecomposeWeightedNorm(torch.autograd.Function):
    """L(G) = sum over the batch and n of w_n |c_n(G)|^2, returned with c (not differentiable):
    forward is one fused decomposition + norm kernel, backward one composition of 2 g w c
    (dL/dG = 2^-N compose(2 g w c), the factor 2 folded into the exact scale 2^(1-N))."""

    @staticmethod
    def forward(ctx, G: torch.Tensor, w: torch.Tensor, method="auto"):
        c, loss = pauli_decompose_weighted_norm(G.contiguous(), w, method=method)
        ctx.save_for_backward(c, w)
        ctx.mark_non_differentiable(c)
        ctx.set_materialize_grads(False)  # no zero-filled gradient for c (a full pass over c)
        return loss, c

    @staticmethod
    def backward(ctx, g: torch.Tensor, _grad_c):
        c, w = ctx.saved_tensors
        N = _qubits_of_coeffs(c)
        if g is None:
            return None, None, None
        g = g.contiguous()
        if N <= 12:
            return pauli_compose_weighted(c, w, g, scale_exp=1 - N), None, None
        return pauli_compose(pauli_weighted_norm_grad(c, w, g), scale_exp=-N), None, None


def decompose_weighted_norm_autograd(G: torch.Tensor, w: torch.Tensor, method="auto"):
    """(L, c) with L differentiable with respect to G."""
    return PauliDecomposeWeightedNorm.apply(G, w, method)


VARIANTS = {"default": 0, "unit8192": 1, "unit4096": 2, "unit4096x8": 3, "unit8192x8": 4, "tiled8": 5,
            "tiled16": 6, "twostage": 7}


OPS = {"decompose": 0, "compose": 1, "decompose_batched": 2, "compose_batched": 3}


def set_variant(N: int, dtype: torch.dtype, op: str, variant) -> None:
    """Select the XOR-diagonal launch shape for (N, dtype, op in OPS); the "_batched" ops set the
    shape used for calls with more than one matrix."""
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    check(_lib.load().pauli_set_variant(int(N), _DTYPES[dtype], OPS[op], v))


def get_variant(N: int, dtype: torch.dtype, op: str) -> int:
    return int(_lib.load().pauli_get_variant(int(N), _DTYPES[dtype], OPS[op]))


def stream_status(stream: torch.cuda.Stream | None = None) -> None:
    """Synchronise the stream and raise PauliError if a tiled launch on it timed out."""
    s = stream if stream is not None else torch.cuda.current_stream()
    check(_lib.load().pauli_stream_status(ctypes.c_void_p(s.cuda_stream)))


def last_error() -> str:
    return _lib.load().pauli_last_error().decode(errors="replace")


def version() -> int:
    return int(_lib.load().pauli_version())


def debug_fail_next_launches(count: int) -> None:
    _lib.load().pauli_debug_fail_next_launches(int(count))


def debug_stall_next_tiled() -> None:
    """Test hook: the next tiled launch gives up on a bounded device wait (PAULI_ERR_TIMEOUT)."""
    _lib.load().pauli_debug_stall_next_tiled()


# short aliases
decompose = pauli_decompose
compose = pauli_compose
coeffs_at = pauli_coeffs_at
decompose_list = pauli_decompose_list
compose_batched = pauli_compose_batched
xhi_layout = pauli_xhi_layout
decompose_xhi = pauli_decompose_xhi
decompose_ws = pauli_decompose_ws
decompose_workspace_size = pauli_decompose_workspace_size
decompose_host = pauli_decompose_host
decompose_host_stream = pauli_decompose_host_stream
decompose_hermitian = pauli_decompose_hermitian
decompose_real = pauli_decompose_real
weighted_norm = pauli_weighted_norm
decompose_weighted_norm = pauli_decompose_weighted_norm
compose_weighted = pauli_compose_weighted
weighted_norm_grad = pauli_weighted_norm_grad
