"""GB300-native dense Pauli decomposition (arXiv 2401.16378): c_n = 2^-N Tr(P_n G) for all
4^N Pauli tensors of a dense 2^N x 2^N complex matrix, and its inverse.

The computation lives in libpauli.so (hand-written CUDA for sm_103a, C ABI in
include/pauli.h); this package is the thin binding. ``workloads`` holds the seeded synthetic
inputs and imports nothing else from the package.
"""
from .api import (PauliDecompose, PauliDecomposeWeightedNorm, PauliError, PauliPlan,  # noqa: F401
                  PauliWeightedNorm, coeffs_at, compose, compose_weighted, debug_fail_next_launches,
                  debug_stall_next_tiled, decompose, decompose_autograd, decompose_hermitian, decompose_host,
                  decompose_host_stream, decompose_list, decompose_real, decompose_weighted_norm,
                  decompose_weighted_norm_autograd, get_variant, last_error, pauli_coeffs_at, pauli_compose,
                  pauli_compose_weighted, pauli_decompose, pauli_decompose_hermitian, pauli_decompose_host,
                  pauli_decompose_host_stream, pauli_decompose_list, pauli_decompose_real,
                  pauli_decompose_weighted_norm, pauli_weighted_norm, pauli_weighted_norm_grad, set_variant,
                  stream_status, version, weighted_norm, weighted_norm_autograd, weighted_norm_grad)
from .api import (compose_batched, decompose_workspace_size, decompose_ws, pauli_decompose_workspace_size,  # noqa: F401
                  pauli_compose_batched, pauli_decompose_ws, release_workspaces, workspace_status)
from .api import decompose_xhi, pauli_decompose_xhi, pauli_xhi_layout, xhi_layout  # noqa: F401
