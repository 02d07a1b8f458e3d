/*
 * pauli.h -- C ABI of libpauli: dense Pauli decomposition and composition on one GB300.
 *
 * Method: T. Jones, "Decomposing dense matrices into dense Pauli tensors", arXiv 2401.16378.
 *
 * Notation (Sec. 2 of the paper): N qubits, D = 2^N. G is a D x D complex matrix, element
 * [G]_{ij} with row i and column j counted from zero. A Pauli tensor index n in [0, 4^N) has
 * base-4 digits p_t = (n >> 2t) & 3 naming operator t as I, X, Y, Z (0, 1, 2, 3); operator 0 is
 * the rightmost Kronecker factor (Sec. 2 first and last paragraphs, Eq. (2)). The coefficients
 * are c_n = 2^-N Tr(P_n G) (Eq. (4)), and G = sum_n c_n P_n (Eq. (1)).
 *
 * Common conventions of every entry point
 *   - Pointers named G, c, out, G_out are DEVICE pointers owned by the caller, unless the
 *     name ends in _host. The library never frees them and keeps no reference after return.
 *   - Matrices are row-major D x D, interleaved complex: complex128 = two float64 (re, im),
 *     complex64 = two float32. Element (r, q) of matrix k of a contiguous batch is at index
 *     k * D * D + r * D + q. Coefficient vectors hold 4^N complex values in the order n.
 *   - Alignment: 16 bytes for complex128 buffers, 8 bytes for complex64.
 *   - Inputs and outputs must not overlap (PAULI_ERR_ALIAS).
 *   - stream is a cudaStream_t passed as void* (NULL = the legacy default stream). Calls are
 *     asynchronous: they validate their arguments, enqueue their kernels and return. Argument
 *     errors are found before anything is enqueued; launch failures map to PAULI_ERR_CUDA.
 *     A fault during execution appears at the caller's next synchronisation.
 *   - Every entry point returns a pauli_status; on failure pauli_last_error() returns a
 *     message for the calling thread. No C++ exception crosses this interface.
 *   - Non-finite input (Inf, NaN) yields NaN in every output that depends on it. Subnormal
 *     inputs of the complex128 XOR-diagonal path are read as zero.
 *   - Arithmetic. complex128: the XOR-diagonal path transforms exact int64 fixed-point values
 *     at a per-XY-mask power-of-two scale; the plain path sums in FP64. complex64: compensated
 *     FP32 -- the XOR-diagonal path splits every value error-free into a high part on a per-mask
 *     power-of-two grid, whose sums are exact, and a low part that carries the rounding errors
 *     (a mask whose values exceed about 2^(126 - N) in magnitude would leave the FP32 range and
 *     gets NaN outputs); the plain path and the norms use TwoSum-compensated FP32 sums.
 */
#ifndef PAULI_H
#define PAULI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { PAULI_C64 = 0, PAULI_C128 = 1 } pauli_dtype;

/* PAULI_PLAIN: the paper's per-coefficient sum, Eq. (13), O(2^N) work per coefficient and
 *   O(8^N) in total (Sec. 3), with the sum index visited in Gray-code order and the sign
 *   updated one bit at a time (Eq. (14)).
 * PAULI_XORDIAG: gathers, for each XY-mask x (Eq. (11)), the XOR-diagonal d_x[i] = G[i^x, i]
 *   and evaluates all 2^N sums that share x at once with a Walsh-Hadamard transform over
 *   the Z/Y mask, O(N 2^N) work per x and O(N 4^N) in total. Same result as Eq. (13).
 * PAULI_AUTO: PAULI_XORDIAG when available for N and dtype, else PAULI_PLAIN. */
typedef enum { PAULI_AUTO = 0, PAULI_PLAIN = 1, PAULI_XORDIAG = 2 } pauli_method;

typedef enum {
  PAULI_OK = 0,
  PAULI_ERR_ARG = 1,      /* N, count, method or another value out of range             */
  PAULI_ERR_NULL = 2,     /* a required pointer is NULL                                  */
  PAULI_ERR_ALIGN = 3,    /* a buffer is not aligned to its element size                 */
  PAULI_ERR_ALIAS = 4,    /* input and output buffers overlap                            */
  PAULI_ERR_DTYPE = 5,    /* dtype is not PAULI_C64 or PAULI_C128                        */
  PAULI_ERR_NOMEM = 6,    /* a plan could not allocate its device memory                 */
  PAULI_ERR_CUDA = 7,     /* a CUDA call failed (launch, copy, device query)             */
  PAULI_ERR_TIMEOUT = 8,  /* a bounded device-side wait gave up (plans, tiled kernel)    */
  PAULI_ERR_UNSUPPORTED = 9 /* valid request this build does not implement (e.g. method) */
} pauli_status;

/* Largest N accepted by the entry points below (memory limits N first: at N = 16 a
 * complex128 matrix is 64 GiB). */
#define PAULI_MAX_QUBITS 16

/* Decompose `count` matrices of N qubits (1 <= N <= PAULI_MAX_QUBITS, count >= 1) stored
 * contiguously at G into 4^N coefficients each, stored contiguously at out.
 *   out[k * 4^N + n] = c_n of matrix k = 2^-N Tr(P_n G_k)              Eq. (4), via Eq. (13).
 * dtype applies to both G and out. method: pauli_method.
 * With PAULI_XORDIAG at N = 12..14 the built-in launch shape is a two-stage one (see
 * PAULI_VARIANT_TWOSTAGE below) that needs a scratch ring between its two stages. This entry point
 * takes it from a library-owned buffer per (device, stream), allocated with cudaMalloc at the
 * first tiled call on that pair, sized for every N so that it is never replaced, and kept until
 * pauli_release_workspaces: make the first such call on a stream before capturing that stream
 * into a CUDA graph. Callers that own their memory use pauli_decompose_ws instead. */
int pauli_decompose(const void* G, int N, int count, int dtype, void* out, int method, void* stream);

/* Bytes of caller-provided scratch that pauli_decompose_ws needs for these arguments (with the
 * launch shape currently chosen for N, dtype and count; see pauli_set_variant), written to
 * *bytes: 0 when the call needs none, else the tiled kernel's scratch ring (tens of MiB). */
int pauli_decompose_workspace_size(int N, int count, int dtype, int method, size_t* bytes);

/* pauli_decompose with the scratch supplied by the caller: the library allocates nothing.
 * workspace: device memory of workspace_bytes >= pauli_decompose_workspace_size(...) bytes,
 * 256-byte aligned, not overlapping G or out (NULL allowed when the size is 0). Its contents
 * need no initialisation; the call clears its control block on `stream` before the launch.
 * One call at a time per workspace: calls that share a workspace must be ordered (one stream,
 * or events). The call can be captured in a CUDA graph. pauli_workspace_status reports the
 * call's device status. Same results, bit for bit, as pauli_decompose. */
int pauli_decompose_ws(const void* G, int N, int count, int dtype, void* out, int method, void* workspace,
                       size_t workspace_bytes, void* stream);

/* Synchronises `stream` and reports (then clears) the status word in a caller workspace of
 * pauli_decompose_ws: PAULI_OK, or PAULI_ERR_TIMEOUT when a bounded wait between the tiled
 * kernel's two stages gave up (that call's results are not valid). */
int pauli_workspace_status(void* workspace, void* stream);

/* Synchronises `stream` and frees the library-owned buffers of the current device for that
 * stream (the tiled decomposition's scratch ring, the weighted norm's partials). Call it before
 * destroying a stream that library calls used; a later call on the stream allocates afresh. */
int pauli_release_workspaces(void* stream);

/* Decomposition of Hermitian matrices: only the real parts are stored,
 *   out_re[k * 4^N + n] = Re c_n of matrix k                                  Eq. (4), (13).
 * Every P_n is Hermitian, so Tr(P_n G^H) is the conjugate of Tr(P_n G): for a Hermitian G every
 * c_n is real and out_re holds all of it; for any G, out_re holds the coefficients of the
 * Hermitian part (G + G^H) / 2. Halves the output bytes and the output conversion.
 *   out_re: device, count * 4^N reals -- double for PAULI_C128, float for PAULI_C64, aligned
 *   to 8 / 4 bytes; must not overlap G.
 * Same methods, kernels and arithmetic as pauli_decompose, so each value is bit for bit the
 * real part that pauli_decompose stores with the same launch shape. Launch shape: the tiled
 * kernel where the decomposition's chosen variant is PAULI_VARIANT_TILED8/16 (N = 12..14;
 * the same scratch buffer), else the single-pass kernel with units of the chosen variant's
 * size (8192 or 4096 elements; always 4096 at N = 6) and 16 elements per thread. */
int pauli_decompose_hermitian(const void* G, int N, int count, int dtype, void* out_re, int method, void* stream);

/* The same for matrices known to be Hermitian, read from the upper triangle only: the real
 * parts of the diagonal and the elements above it (q > r). The strict lower triangle is never
 * read and the diagonal's imaginary parts are never used: both may hold anything.
 *   out_re[k * 4^N + n] = c_n of the Hermitian matrix with that upper triangle   Eq. (4), (13).
 * For an XY-mask x != 0 with top set bit h the XOR-diagonal satisfies e_x[r ^ x] = conj(e_x[r]);
 * the rows with bit h clear are exactly the upper-triangle elements of the class, and one
 * Walsh-Hadamard transform over the other N - 1 row bits gives two real coefficients per
 * value: c(x, z) = 2^(1-N) Re(V[z without bit h] i^popc(x & z)) for z_h = 0 and 1. So the
 * XOR-diagonal kernel reads half of G and writes reals: 16 bytes per complex128 coefficient
 * instead of 32. The XOR-diagonal kernel covers N 7..12; at N = 13, 14 (PAULI_AUTO or
 * PAULI_XORDIAG; count <= 1024, G 16-byte aligned) the two-stage kernel runs in an
 * upper-triangle mode: a 64 x 64 tile below the diagonal is loaded from its mirror above and
 * read transposed and conjugated, diagonal tiles mirror their own lower halves, so half of G is
 * read (the full transform is still computed) and reals are written; for Hermitian G the
 * values equal pauli_decompose_hermitian's in the same launch shape bit for bit. Smaller N and
 * PAULI_PLAIN take the per-coefficient sum with the lower triangle read through its mirror;
 * N > 14 is PAULI_ERR_UNSUPPORTED. Arguments as for pauli_decompose_hermitian. */
int pauli_decompose_hermitian_upper(const void* G, int N, int count, int dtype, void* out_re, int method,
                                    void* stream);

/* Decomposition of real matrices. G_real: `count` row-major D x D float64 matrices (8 bytes per
 * element; dtype must be PAULI_C128, PAULI_ERR_UNSUPPORTED otherwise). For real G every
 * XOR-diagonal is real and so is its Walsh-Hadamard transform, so c_n is real when P_n has an
 * even number k of Y factors and imaginary when k is odd (each Y entry is imaginary, Eq. (3)).
 * out_re: count * 4^N float64, the real number a_n with c_n = i^(k mod 2) a_n, that is
 * Re c_n for even k and Im c_n for odd k. Reads 8 and writes 8 bytes per coefficient instead of
 * 16 and 16. Same kernels and launch shapes as pauli_decompose (complex128 arithmetic with zero
 * imaginary parts), so a_n equals, bit for bit, the nonzero part that pauli_decompose stores for
 * G + 0i with the same launch shape. */
int pauli_decompose_real(const void* G_real, int N, int count, int dtype, void* out_re, int method, void* stream);

/* Compose: G_out[k] = 2^scale_exp * sum_n c[k * 4^N + n] P_n                         Eq. (1).
 * scale_exp in [-64, 64] is an exact power-of-two factor; scale_exp = -N gives the adjoint
 * of pauli_decompose (the gradient of a real loss with respect to G is
 * 2^-N compose(grad_c), because every P_n is Hermitian). */
int pauli_compose(const void* c, int N, int count, int dtype, void* G_out, int scale_exp, void* stream);

/* Weighted norm of `count` coefficient vectors, a real loss of the decomposition:
 *   *loss = sum_{k < count} sum_{n < 4^N} w_n |c[k * 4^N + n]|^2.
 * With w = 1 and c = decompose(G) it equals 2^-N ||G||_F^2, since Tr(P_m P_n) = 2^N [m = n]
 * (the Pauli tensors of Sec. 2 are Hermitian, unitary and trace-orthogonal).
 *   c: device, count * 4^N complex values of dtype. w: device, 4^N reals -- double for
 *   PAULI_C128, float for PAULI_C64. loss: device, one real of that type, overwritten.
 * FP64 accumulation for PAULI_C128; compensated FP32 per thread and FP64 across threads for
 * PAULI_C64. The summation order is fixed, so repeated calls give identical bits. Uses an
 * 8 KiB device workspace per (device, stream), allocated with cudaMalloc at the first call
 * on that pair and kept: make the first call before capturing the stream in a CUDA graph.
 * loss must not overlap c or w (PAULI_ERR_ALIAS). */
int pauli_weighted_norm(const void* c, int N, int count, int dtype, const void* w, void* loss, void* stream);

/* Gradient of pauli_weighted_norm's loss with respect to c, in PyTorch's convention for a
 * real function of complex inputs (dL/dRe c + i dL/dIm c), times the incoming gradient g:
 *   grad_c[k * 4^N + n] = 2 g w_n c[k * 4^N + n].
 * g: device pointer to one real of the loss's type, or NULL for g = 1. grad_c: device, same
 * size and dtype as c; grad_c == c (in place) is allowed, any other overlap of grad_c with c,
 * w or g is PAULI_ERR_ALIAS. Chained with pauli_compose(grad_c, scale_exp = -N) it gives the
 * gradient of the loss with respect to G. Allocates nothing. */
int pauli_weighted_norm_grad(const void* c, int N, int count, int dtype, const void* w, const void* g,
                             void* grad_c, void* stream);

/* Fused forward step of that loss: pauli_decompose(G -> out) and pauli_weighted_norm(out -> loss)
 * in one pass over G for N = 6..12 with the XOR-diagonal method (the decomposition kernel adds
 * w_n |c_n|^2 over the coefficients it stores; one FP64 partial per work unit, added in a fixed
 * order, so the loss is deterministic); for other N, or PAULI_PLAIN, the two calls in sequence.
 * Arguments as in those two calls; out, w and loss must not overlap each other or G. Uses the
 * per-(device, stream) workspace of pauli_weighted_norm, grown to 8 bytes per 4096 elements of
 * the batch at the first call that needs more (cudaMalloc; not while capturing a graph). */
int pauli_decompose_weighted_norm(const void* G, int N, int count, int dtype, void* out, const void* w,
                                  void* loss, int method, void* stream);

/* Composition of weighted coefficients:
 *   G_out[k] = 2^scale_exp * sum_n g w_n c[k * 4^N + n] P_n                           Eq. (1).
 * One pass over c: each loaded c_n is multiplied by g w_n (one rounding) before the transform.
 * w: device, 4^N reals (double for PAULI_C128, float for PAULI_C64); g: device pointer to one
 * such real, or NULL for 1. With scale_exp = 1 - N this is the gradient of
 * pauli_weighted_norm's loss with respect to G, 2^-N compose(2 g w c), bit for bit equal to
 * pauli_weighted_norm_grad followed by pauli_compose(scale_exp = -N) with the same launch shape.
 * N <= 12 (PAULI_ERR_UNSUPPORTED above). */
int pauli_compose_weighted(const void* c, int N, int count, int dtype, const void* w, const void* g, void* G_out,
                           int scale_exp, void* stream);

/* Coefficients for a caller-chosen list of indices: out[q] = c_{idx[q]} for q < k, each by
 * the per-coefficient sum of Eq. (13) in O(2^N) work and no scratch memory -- the use the
 * paper's fixed-memory property is for (abstract; Sec. 3). idx is a device array of k
 * uint64 values < 4^N (values out of range yield NaN); out holds k complex values. */
int pauli_coeffs_at(const void* G, int N, int dtype, const uint64_t* idx, int64_t k, void* out, void* stream);

/* Separate launches over a list of matrices of different N: G_list[b] and out_list[b] are
 * host arrays of device pointers, N_list a host array; one pauli_decompose (count = 1,
 * the given method) per entry, in order, on the same stream. Allocates nothing. */
int pauli_decompose_list(const void* const* G_list, const int* N_list, int batch, int dtype,
                         void* const* out_list, int method, void* stream);

/* Composition of a batch of coefficient vectors of uneven N in one launch (per 1024 matrices):
 *   G_out_list[b] = 2^scale_exp * sum_n c_list[b][n] P_n          Eq. (1), for every b < batch.
 * c_list[b]: device, 4^N_b coefficients in the order n; G_out_list[b]: device, the 2^N_b x 2^N_b
 * matrix; the two host arrays hold device pointers, N_list is a host array of values in
 * [1, 11]; scale_exp in [-64, 64] (scale_exp = -N_b gives the adjoint of the decomposition, when
 * every N_b is equal). For N_b >= 6 each 4096-element XOR-diagonal unit is one work item (the
 * transform of Eq. (1) over the Z/Y mask for 2^(12-N_b) XY-masks); smaller matrices are one
 * item each. The matrix table is passed to the kernel by value and its CTAs take the items in a
 * fixed order, so the call allocates nothing, keeps no state between calls, returns without
 * waiting for the GPU and can be captured in a CUDA graph. Same arithmetic as pauli_compose
 * (complex128: exact int64 transform of each XY-mask's values at a per-mask power-of-two scale;
 * complex64: compensated FP32 on per-mask grids). Input and output buffers must not overlap. */
int pauli_compose_batched(const void* const* c_list, const int* N_list, int batch, int dtype,
                          void* const* G_out_list, int scale_exp, void* stream);

/* x-class shards. Every XY-mask x of Eq. (13) is an independent transform (Sec. 3 notes that the
 * coefficients can be evaluated independently and distributed), so the 2^N classes can be split
 * over 2^k devices by their top k bits x_hi. With m = N - k, the shard x_hi needs only the 2^k
 * blocks of G (2^m x 2^m, at block row r_hi and block column r_hi ^ x_hi; r_hi = r >> m):
 *   c(x, z) = 2^-k i^popc(x_hi & z_hi) sum_{r_hi} (-1)^popc(r_hi & z_hi) c_{B(r_hi)}(x_lo, z_lo),
 * B(r_hi) the m-qubit block, x = (x_hi, x_lo), z = (z_hi, z_lo) split at bit m, and c_B(n_lo) the
 * block's own coefficients, whose index n_lo = n(x_lo, z_lo) is the low 2m bits of n(x, z).
 *
 * Block-XOR layout L of the shard: D rows of 2^m elements, the blocks stacked by r_hi:
 *   L[r * 2^m + j] = G[r, ((r_hi ^ x_hi) << m) | j],   0 <= r < D, 0 <= j < 2^m,
 * 4^N / 2^k elements of dtype. pauli_xhi_layout builds it from a full device G (one copy kernel
 * on the stream); a row-sharded G reaches it with one all-to-all, in which device w sends
 * its block column w ^ g to device g.
 *   G: device, D x D row-major; L: device, 4^N / 2^k elements; 0 <= k <= N - 1,
 *   0 <= x_hi < 2^k; G and L must not overlap. */
int pauli_xhi_layout(const void* G, int N, int k, int x_hi, int dtype, void* L, void* stream);

/* The coefficients of the shard x_hi from its block-XOR layout L (above):
 *   out[(z_hi << 2m) | n_lo] = c_n,  n = n_lo | (spread(x_hi ^ z_hi) | spread(z_hi) << 1) << 2m,
 * for z_hi < 2^k and n_lo < 4^m (spread: bit t to bit 2t), 4^N / 2^k elements of dtype.
 * For N = 12..14 with m >= 6 and PAULI_AUTO / PAULI_XORDIAG (L 16-byte aligned): one launch
 * of the two-stage kernel over the shard's classes, reading L's tiles and writing the compact
 * order directly, bit for bit the values pauli_decompose gives for those coefficients with its
 * two-stage shape (the scratch of pauli_decompose). Otherwise: one pauli_decompose of the 2^k
 * blocks (m qubits, count 2^k, the given method) into out, then, in place, the k-bit
 * Walsh-Hadamard transform over r_hi with the phase and the exact scale 2^-k, in passes of up
 * to 4 bits (FP64 sums for both dtypes; complex64 rounds once per pass). The shards' outputs
 * together hold every c_n once; k = 0 is pauli_decompose. L and out must not overlap. */
int pauli_decompose_xhi(const void* L, int N, int k, int x_hi, int dtype, void* out, int method, void* stream);

/* Host-buffer round trip for callers whose data is in host memory: copies `count` matrices
 * from G_host (pinned memory gives asynchronous copies) to the caller's device buffer G_dev,
 * decomposes into out_dev, and copies the coefficients back to out_host, all on `stream`.
 * The call returns after enqueueing; the host buffers must stay valid until the stream has
 * finished. */
int pauli_decompose_host(const void* G_host, int N, int count, int dtype, void* out_host, void* G_dev,
                         void* out_dev, int method, void* stream);

/* Streams a list of host matrices of one N through the device: matrix k is copied in from
 * G_host_list[k], decomposed (method as for pauli_decompose) and its 4^N coefficients copied out
 * to out_host_list[k]. The work is pipelined over two caller-owned device buffer pairs
 * (G_dev[0..1], out_dev[0..1]: device arrays of 4^N elements each, all four distinct) and three
 * library streams -- copy in, compute, copy out -- ordered by events, so that the copy-in of
 * matrix k + 1, the decomposition of matrix k and the copy-out of matrix k - 1 proceed at once
 * (both directions of the host link and the SMs busy together). The pipeline starts after
 * earlier work on `stream`, and later work on `stream` waits for its last copy; the call
 * returns after enqueueing. Host buffers should be pinned (else the copies are synchronous)
 * and stay valid until the stream has finished. G_host_list, out_host_list: host arrays of
 * n_mats host pointers (an input may repeat); G_dev, out_dev: host arrays of 2 device pointers.
 * The library's streams and events are created at the first call on each device and kept;
 * calls on one device enqueue one at a time. */
int pauli_decompose_host_stream(const void* const* G_host_list, void* const* out_host_list, int n_mats, int N,
                                int dtype, void* const* G_dev, void* const* out_dev, int method, void* stream);

/* Batched decomposition for callers that cannot allocate device memory (a fixed memory
 * budget, an allocator that must not be re-entered, ...). Same result and same one-launch
 * schedule as a plan over N_list, but the library allocates nothing: the work counter,
 * status word and matrix table live in a fixed array in device global memory that is part of
 * the library image (24,608 bytes on every GPU that loads the library, kept until the process
 * exits). There is no counterpart in the paper; this is an interface convenience.
 *   G_list / out_list: host arrays of `batch` device pointers; N_list: host array, values in
 *   [1, 10]; 1 <= batch <= 1024 (larger batches are rejected with PAULI_ERR_ARG).
 * The call enqueues two kernels and returns without waiting for the GPU: the first receives
 * the matrix table by value (as a kernel parameter), writes it to the array and clears the
 * counter and status; the second decomposes. The host arrays may be reused as soon as the call
 * returns.
 * All calls share the array and it keeps the last call's contents; calls whose kernels overlap
 * on the GPU race on it -- serialise them (one stream, or events). The first call on a device
 * looks up the array's device address; make it before any stream capture. */
int pauli_decompose_batch_static(const void* const* G_list, const int* N_list, int batch, int dtype,
                                 void* const* out_list, void* stream);

/* ---- Plans: one persistent launch over a batch of matrices of uneven N -------------------
 * A plan fixes the list of N and the dtype, owns a device work list (the matrices' x-class
 * work units ordered by descending cost), a device work counter and a device status word,
 * and chooses its launch shape once (from the autotuner's choice when one is given).
 * pauli_plan_execute enqueues a reset of the counter and ONE kernel launch that decomposes
 * every matrix; it can be captured in a CUDA graph, and pauli_plan_graph_launch does that
 * capture once and replays the graph afterwards.
 *   N_list: host array of batch values in [1, 10]; G_list / out_list: host arrays of device
 *   pointers bound by pauli_plan_bind (copied to the plan's device memory, synchronous). */
typedef struct pauli_plan pauli_plan;

int pauli_plan_create(const int* N_list, int batch, int dtype, int threads_per_block, int blocks_per_sm,
                      pauli_plan** plan);
/* A plan for Hermitian matrices: each execution decomposes the bound matrices read from their
 * upper triangle (as pauli_decompose_hermitian_upper: the strict lower triangle and the
 * diagonal's imaginary parts are never used) and stores real coefficients, out_list[b] holding
 * 4^N reals (double for PAULI_C128, float for PAULI_C64). Matrices from N = 7 (N = 6 with
 * threads_per_block = 256) are cut into upper-triangle units over half the rows; smaller ones
 * are one item each. Everything else as for pauli_plan_create. */
int pauli_plan_create_hermitian(const int* N_list, int batch, int dtype, int threads_per_block, int blocks_per_sm,
                                pauli_plan** plan);
int pauli_plan_bind(pauli_plan* plan, const void* const* G_list, void* const* out_list);
int pauli_plan_execute(pauli_plan* plan, void* stream);
int pauli_plan_graph_launch(pauli_plan* plan, void* stream);
/* Synchronises the plan's last stream and reports its device status word: PAULI_OK, or
 * PAULI_ERR_TIMEOUT when a bounded wait in the kernel gave up. */
int pauli_plan_status(pauli_plan* plan);
/* Test hook: 1 makes the next execution wait on a flag that nothing sets; the wait gives up
 * after a bounded number of polls and records PAULI_ERR_TIMEOUT. 0 restores normal runs. */
int pauli_plan_set_stall(pauli_plan* plan, int stall);
void pauli_plan_destroy(pauli_plan* plan);

/* ---- Launch-shape variants of PAULI_XORDIAG ----------------------------------------------
 * PAULI_VARIANT_UNIT8192:   8192-element work units, 512-thread CTAs (16 elements per thread,
 *                           one CTA per SM), N 7..15.
 * PAULI_VARIANT_UNIT4096:   4096-element work units, 256-thread CTAs (16 per thread, two CTAs
 *                           per SM), N 6..14.
 * PAULI_VARIANT_UNIT4096X8: 4096-element work units, 512-thread CTAs (8 per thread, two CTAs
 *                           per SM), N 6..14.
 * PAULI_VARIANT_UNIT8192X8: 8192-element work units, 1024-thread CTAs (8 per thread), N 7..15.
 * For N above 12 (resp. 11) a unit is one pair of XY-masks spread over a CTA cluster.
 * PAULI_VARIANT_TILED8:     decomposition only, N 12..14, count <= 1024, G 16-byte aligned:
 *                           two stages through a library-owned scratch ring that stays in L2.
 *                           Stage 1 reads tiles of 64 XY-masks x 64 rows (each row a contiguous
 *                           64-element run of G) and does the 6 low transform stages; stage 2
 *                           the other N - 6. One persistent, warp-specialised launch (a copy
 *                           warp feeding 512 compute threads, 8 elements each, through a ring
 *                           of shared-memory buffers). The scratch (S x 2^(N+10) bytes plus
 *                           a little, S = 6, 5, 3 slots at N = 12, 13, 14) comes from the
 *                           library's buffer for the (device, stream) pair, or from the caller
 *                           (pauli_decompose_ws). Calls on one stream are ordered by the stream;
 *                           calls on different streams get different library buffers.
 * PAULI_VARIANT_TILED16:    the same with two groups of 256 compute threads of 16 elements
 *                           each, working on alternate buffers.
 * PAULI_VARIANT_TWOSTAGE:   decomposition only, N 12..14 (the built-in choice there): the
 *                           same two stages, tiles and scratch ring, with every compute warp
 *                           running its 512 elements of a work item on its own (its own part of
 *                           the tile, its own copy of the stage-2 data, exchanges within the warp)
 *                           and no barrier between the warps of an item. complex64 runs compensated
 *                           FP32: each value split into a high part on a per-mask power-of-two
 *                           grid, whose sums are exact, and a low part that carries the rounding
 *                           errors (error-free Fast2Sum against the grid's anchor); between the
 *                           stages each value is kept as one float per part (8 bytes: the pair
 *                           rounded once) and split again on the whole mask's grid. Scratch as
 *                           for the tiled variants (complex64 uses half of it);
 *                           pauli_decompose_workspace_size reports it.
 * All variants compute bit-identical complex128 results, except that the two-stage ones re-scale
 * partial sums between the stages (an extra truncation below the class quantum, well inside
 * the accuracy bound of pauli_decompose; the three two-stage variants agree with each other bit
 * for bit); they differ otherwise only in speed. complex64 results of different variants agree
 * to within the accuracy bound, not bit for bit. The choice is
 * process-wide per (N, dtype, op): op 0 = decompose, 1 = compose, for calls on one matrix
 * (count = 1); op 2 = decompose, 3 = compose, for calls on a batch (count > 1), where the
 * units of many matrices fill the GPU and a different shape can win. Variant 0 restores the
 * built-in default. The autotuner in the Python package measures the variants and records
 * its choice here. */
#define PAULI_VARIANT_DEFAULT 0
#define PAULI_VARIANT_UNIT8192 1
#define PAULI_VARIANT_UNIT4096 2
#define PAULI_VARIANT_UNIT4096X8 3
#define PAULI_VARIANT_UNIT8192X8 4
#define PAULI_VARIANT_TILED8 5
#define PAULI_VARIANT_TILED16 6
#define PAULI_VARIANT_TWOSTAGE 7
int pauli_set_variant(int N, int dtype, int op, int variant);
/* The variant in effect for (N, dtype, op), or 0 when PAULI_XORDIAG has none for N. */
int pauli_get_variant(int N, int dtype, int op);

/* Synchronises `stream` and reports the status word of the tiled variants' scratch on that
 * stream (then clears it): PAULI_OK, or PAULI_ERR_TIMEOUT when a bounded wait between the two
 * stages gave up since the last call (the results of that launch are not valid). PAULI_OK when
 * no tiled launch has used the stream. */
int pauli_stream_status(void* stream);

/* Message for the last failing call on this thread ("" when none). */
const char* pauli_last_error(void);
/* Library version as MAJOR * 10000 + MINOR * 100 + PATCH. */
int pauli_version(void);
/* Test hook for the host error path: when nonzero, the next `count` launches report
 * PAULI_ERR_CUDA as if the launch had failed, without enqueueing anything. */
void pauli_debug_fail_next_launches(int count);
/* Test hook for the device timeout path of the tiled variants: the next tiled launch makes its
 * producers wait (a few milliseconds, bounded) on a count that nothing raises; they give up,
 * record PAULI_ERR_TIMEOUT for pauli_stream_status and end the launch early (its output is
 * then not valid). */
void pauli_debug_stall_next_tiled(void);

#ifdef __cplusplus
}
#endif

#endif /* PAULI_H */
