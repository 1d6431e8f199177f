/*
 * qk.h -- C ABI of libqk.so: structured-Gram kernel solves over randomized
 * low-discrepancy points on one GB300 (sm_103a).
 *
 * The operations follow arXiv 2502.14256 ("QMCPy ... randomized LD sequences,
 * ... fast kernel methods"):
 *   points     Sec. 4.2 (shifted rank-1 lattices, natural order, base 2) and
 *              Sec. 4.3 (base-2 digital nets, Matousek linear matrix scrambling,
 *              digital shift, natural or Gray-code order);
 *   kernels    Sec. 5.2 Eq. (K_SI_prod) (shift-invariant Bernoulli kernels with
 *              product weights) and Sec. 5.3 Eq. (DSI kernel) with the closed
 *              forms of the Theorem there (digitally-shift-invariant kernels);
 *   spectra    Sec. 5.4: K = V diag(lambda) V^H, lambda = sqrt(n) conj(V) k_1,
 *              K y = V(y~ * lambda), K^-1 y = V(y~ / lambda), with V = H/sqrt(n)
 *              (Hadamard, FWHT) for nets and the bit-reversed Fourier matrix
 *              (FFTBR / IFFTBR) for lattices;
 *   MLL        Sec. 3.2 (kernel interpolation / GP hyper-parameter fitting and the
 *              kernel discrepancy with kappa_i = int K(u, x_i) du); the gradient is
 *              the textbook GP gradient carried through the spectrum.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, unless a comment
 *     says "host".  The library allocates no device memory: scratch space comes
 *     from a caller-provided workspace whose size qk_workspace_bytes() returns.
 *   - Every call is asynchronous on the given stream (NULL = legacy default
 *     stream) and returns a qk_status.  Argument errors are detected on the host
 *     before any launch (QK_EINVAL) and nothing is launched.  A CUDA launch error
 *     returns QK_ECUDA.  Conditions only the device can see (a non-positive
 *     eigenvalue, a bounded wait that expired) are OR-ed into the optional
 *     device status word `status` (bits QK_STATUS_*); qk_read_status() turns it
 *     into a qk_status after synchronising the stream.
 *   - qk_last_error() copies a message describing the last failure on the
 *     calling host thread.
 *   - Points are 32-bit words: coordinate x = X * 2^-32 (t_max = 32 digits; the
 *     first digit is bit 31).
 *   - n = 2^m with 0 <= m <= QK_MAX_M, 1 <= d <= QK_MAX_D.
 */
#ifndef QK_H
#define QK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *qk_stream; /* same type as cudaStream_t */

#if defined(__GNUC__)
#define QK_API __attribute__((visibility("default")))
#else
#define QK_API
#endif

enum qk_status {
  QK_OK = 0,
  QK_EINVAL = 1,     /* bad argument (size, null pointer, alignment, enum value) */
  QK_ENOTPD = 2,     /* some eigenvalue <= 0: K is not positive definite */
  QK_ECUDA = 3,      /* a CUDA runtime call or launch failed */
  QK_ETIMEOUT = 4,   /* a bounded device-side wait expired */
  QK_EWORKSPACE = 5  /* workspace null or smaller than qk_workspace_bytes() */
};

/* QK_STATUS_FLOOR is informational: some computed eigenvalue fell below the nugget
 * eta > 0 and was raised to eta (the spectrum of K + eta I lies in [eta, inf), so a
 * smaller value can only be rounding, e.g. FP32 transforms at large n).
 * qk_read_status reports it as QK_OK. */
enum qk_status_bits { QK_STATUS_NOTPD = 1u, QK_STATUS_TIMEOUT = 2u, QK_STATUS_FLOOR = 4u };

enum qk_kind { QK_NET_B2 = 0, QK_LATTICE = 1 };
enum qk_order { QK_NATURAL = 0, QK_GRAY = 1 };
enum qk_family { QK_DSI = 0, QK_SI = 1 };
/* QK_F32W: FP32 data and FP32 arithmetic, except that the first column is carried as
 * float-float pairs (about 2^-46 relative per kernel factor, still on the FP32 pipes) and
 * transformed with compensated (float-float) butterflies, so that every eigenvalue is
 * accurate to about 2^-44 lambda_max before it is rounded, instead of eps32 ||k_1||.  Use
 * it when the spectrum reaches far below eps32 lambda_max (a small nugget, many
 * dimensions, large n): there an FP32 column moves the small eigenvalues by more than
 * themselves, and every 1/lambda-weighted output (solve, quadratic form, log det,
 * gradient) inherits that.  Accepted by qk_kernel_col / qk_kernel_col_at (which then
 * write FP64 values) and by the batched schedule (FP32 y and c; the refinement of the
 * FP32 schedule is always on).  Other entry points take QK_F64 or QK_F32 only. */
enum qk_dtype { QK_F64 = 0, QK_F32 = 1, QK_F32W = 2 };
/* Form of a stored first column: the column itself, or p = k_1/zeta - 1
 * (computed by a product-minus-one recurrence, so that the variation of the
 * kernel around its constant part keeps full relative precision). */
enum qk_colform { QK_COL_K1 = 0, QK_COL_P = 1 };

#define QK_MAX_M 30
#define QK_MAX_D 256

/* A randomized point set (Sec. 4.2 / 4.3).  Holds R randomizations. */
typedef struct {
  int32_t kind;        /* QK_NET_B2 or QK_LATTICE */
  int32_t order;       /* nets: QK_NATURAL or QK_GRAY; lattices: QK_NATURAL */
  uint32_t d;          /* dimensions */
  uint32_t R;          /* randomizations stored in Ct / D */
  const uint32_t *Ct;  /* nets: (R, d, 32) scrambled generator columns
                          (qk_lms_setup output); column k, bit 31-t = digit t */
  const uint32_t *g;   /* lattices: (d) generating vector */
  const uint32_t *D;   /* (R, d) shift words: XOR for nets (digital shift),
                          + mod 2^32 for lattices; NULL means no shift */
} qk_pointset;

/* Product-weight kernel K(x,x') = zeta prod_j (1 + c_j K_alpha(x_j, x'_j)). */
typedef struct {
  int32_t family;         /* QK_DSI (nets) or QK_SI (lattices) */
  int32_t alpha;          /* DSI order 1, 2, 3, 4; SI smoothness 1 or 2 */
  uint32_t d;
  const double *weights;  /* (d) effective weights c_j (gamma_j * lengthscale_j) */
  double zeta;            /* scale, > 0 */
} qk_kernel;

/* Per right-hand side result of qk_mll (doubles, in this order). */
#define QK_MLL_QUAD 0      /* y^T K^-1 y */
#define QK_MLL_LOGDET 1    /* log det K */
#define QK_MLL_MLL 2       /* -quad/2 - logdet/2 - n log(2 pi)/2 */
#define QK_MLL_MEAN 3      /* Bayesian-cubature posterior mean zeta 1^T K^-1 y */
#define QK_MLL_VAR 4       /* posterior variance zeta - zeta^2 1^T K^-1 1 */
#define QK_MLL_NOUT 5
/* Gradient block per right-hand side: 2d + 2 doubles:
 *   [0, d)       dMLL/dc_j
 *   d            dMLL/deta
 *   [d+1, 2d+1)  dMEAN/dc_j
 *   2d+1         dMEAN/deta
 * Chain rule to log-lengthscales theta_j (c_j = gamma_j e^theta_j): c_j dMLL/dc_j. */

/* ---------------------------------------------------------------- points --- */

/* Linear matrix scrambling C~_j = S_j C_j over GF(2) (Sec. 4.3, LMS).
 * C: (d, 32) generator columns; S: (R, d, 32) row masks of the scrambling
 * matrices (row t, bit 31-u = entry (t, u)); Ct: (R, d, 32) output. */
QK_API int qk_lms_setup(uint32_t d, uint32_t R, const uint32_t *C, const uint32_t *S,
                 uint32_t *Ct, qk_stream stream);

/* Points of randomizations r0 .. r0+nr-1 at sequence positions i0 .. i0+n-1
 * (any range; Sec. 4.2 "n_min/n_max").  X: (nr, n, d) uint32 row-major.
 * Nets: X = D (+) XOR_{bit k of g(i)} Ct[:, k], g(i) = i or the Gray code of i.
 * Lattices: X = (v(i) 2^32 * g + D) mod 2^32 with v the radical inverse.
 * i0 + n <= 2^32. */
QK_API int qk_gen_points(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0,
                  uint64_t n, uint32_t *X, qk_stream stream);

/* ------------------------------------------------------------ first column --- */

/* First Gram column k_1[i] = K(x_i, x_0) for n = 2^m points of randomizations
 * r0 .. r0+nr-1 (Sec. 5.4, "k1 = kernel(x, x[0])").  The shift cancels in
 * x_i (-) x_0, so only Ct (nets) or g (lattices) is read.  col: (nr, n) in
 * dtype, in the requested form (QK_COL_K1 or QK_COL_P); with QK_F32W, (nr, n) doubles
 * computed in float-float arithmetic. */
QK_API int qk_kernel_col(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr,
                  uint32_t m, int32_t dtype, int32_t form, void *col, qk_stream stream);

/* qk_kernel_col for the 2^m points at positions i0 .. i0 + 2^m - 1 of the same
 * sequence (i0 a multiple of 2048): e.g. the new half of an extended point set, for
 * qk_eigs_extend.  col: (nr, 2^m) in dtype and form. */
QK_API int qk_kernel_col_at(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint64_t i0,
                            uint32_t m, int32_t dtype, int32_t form, void *col, qk_stream stream);

/* ------------------------------------------------------------- spectrum --- */

/* Eigenvalues lambda = sqrt(n) conj(V) k_1 + eta (Sec. 5.4) of `batch` Gram
 * matrices from their first columns col (batch, n) (dtype, form).  DSI: FWHT,
 * lambda in Hadamard order; SI: FFTBR, lambda in frequency order (real).
 * The transform runs in dtype; the nugget, zeta and the sign test in FP64.
 * lam: (batch, n) doubles.  Eigenvalues below eta > 0 are raised to eta
 * (QK_STATUS_FLOOR); with eta <= 0, QK_STATUS_NOTPD is set if some lambda <= 0. */
QK_API int qk_eigs(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form,
            const void *col, double zeta, double eta, double *lam, void *ws,
            size_t ws_bytes, uint32_t *status, qk_stream stream);

/* Eigenvalues exactly as qk_eigs, for callers that cannot allocate device memory
 * at the call site (for instance a plug-in whose host application owns all GPU
 * memory through its own allocator, or a fixed-footprint service that forbids
 * allocations after start-up): no workspace argument, the scratch space is a static
 * device array of QK_EIGS_STATIC_MAX_BYTES owned by the library, held on every GPU
 * that loads it until the process exits.  The paper has no counterpart to this
 * entry point.  Requests needing more scratch than that (batch * 2^m elements of the
 * transform type: 8 bytes for FP64 nets, 4 for FP32 nets, 16 and 8 for lattices)
 * return QK_EINVAL and launch nothing.  The first call on each device looks up the
 * array's device address with that device current; make it before any stream
 * capture.  The address is kept for the life of the process: no call may follow a
 * cudaDeviceReset of that device (the reset unloads the array).  All calls share the
 * array and it keeps the last call's contents (none needs to start at zero); calls
 * whose kernels overlap on the GPU race on it and must be serialised by the caller. */
#define QK_EIGS_STATIC_MAX_BYTES ((size_t)4 << 20)
QK_API int qk_eigs_static(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form,
                          const void *col, double zeta, double eta, double *lam, uint32_t *status,
                          qk_stream stream);

/* Doubling update of the eigenvalues (Sec. 5.4, efficient eigenvalue updates): for a
 * point set extended from n = 2^m to 2n points (its first n points being the n-point
 * set: nets in natural or Gray order, lattices in natural order), the eigenvalues of the
 * 2n-point Gram matrix from those of the n-point matrix and the first-column entries of
 * the n new points only:
 *   lambda' = [lambda + w (.) t, lambda - w (.) t],  t = sqrt(n) conj(V_m) k_new,
 * w_k = 1 (nets) or exp(-pi i k / n) (lattices); one transform of length n instead of 2n.
 * lam_old: (batch, n) doubles from qk_eigs (nugget included); col_new: (batch, n) in
 * dtype and form (qk_kernel_col_at with i0 = n); lam: (batch, 2n) doubles, must not
 * overlap lam_old.  The floor / sign tests of qk_eigs apply to the result.
 * Workspace: qk_workspace_bytes op 0 with (family, m, batch). */
QK_API int qk_eigs_extend(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form,
                          const void *col_new, double zeta, double eta, const double *lam_old, double *lam,
                          void *ws, size_t ws_bytes, uint32_t *status, qk_stream stream);

/* Solve K c = y for `batch` Gram matrices and nrhs right-hand sides each:
 * c = V (y~ / lambda), y~ = conj(V) y (Sec. 5.4).  y, c: (batch, nrhs, n) in
 * dtype (may alias); lam: (batch, n) from qk_eigs.  The division is done in
 * FP64.  refine_steps >= 0 steps of iterative refinement c += K^-1 (y - K c),
 * the residual evaluated with FP64 transforms (meaningful for QK_F32). */
QK_API int qk_solve(int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs, int32_t dtype,
             const double *lam, const void *y, void *c, int32_t refine_steps, void *ws,
             size_t ws_bytes, qk_stream stream);

/* Matrix-vector product u = K y = V (y~ * lambda) (Sec. 5.4). */
QK_API int qk_matvec(int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs, int32_t dtype,
              const double *lam, const void *y, void *u, void *ws, size_t ws_bytes,
              qk_stream stream);

/* Marginal log-likelihood, log det, quadratic form and Bayesian-cubature
 * posterior mean / variance for randomizations r0 .. r0+nr-1 of ps with nrhs
 * right-hand sides each; y: (nr, nrhs, n) dtype; lam: (nr, n) from qk_eigs
 * with the same kernel and eta.  out: (nr, nrhs, QK_MLL_NOUT) doubles.
 * grad (nullable): (nr, nrhs, 2d+2) doubles, the gradient block above,
 * computed by carrying g_w = (|y~_w|^2/lambda_w^2 - 1/lambda_w)/2 back through
 * the transform and recomputing the kernel factors (nothing n x d is stored). */
QK_API int qk_mll(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m,
           uint32_t nrhs, int32_t dtype, double eta, const double *lam, const void *y,
           double *out, double *grad, void *ws, size_t ws_bytes, uint32_t *status,
           qk_stream stream);

/* ------------------------------------------------------------ transforms --- */

/* In-place batched transforms of nvec contiguous vectors of length n = 2^m
 * (Sec. 5.2-5.3; the paper's fwht / fftbr / ifftbr):
 *   qk_fwht:   x <- H_m x / sqrt(n)               (real; dtype elements)
 *   qk_fftbr:  x <- DFT(x taken in linear order) / sqrt(n), x given in natural
 *              (bit-reversed) order, result in frequency order
 *   qk_ifftbr: the inverse of qk_fftbr (frequency order in, natural order out)
 * FFT data are interleaved complex (re, im) pairs of dtype.  Radix-2
 * butterflies (a +- W b)/sqrt(2) as in the paper's FFTBR/FWHT schemes. */
QK_API int qk_fwht(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream);
QK_API int qk_fftbr(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream);
QK_API int qk_ifftbr(uint32_t m, uint64_t nvec, int32_t dtype, void *x, qk_stream stream);

/* Doubling update of transformed data (Sec. 5.4): from xt_old = the transform of the
 * first n = 2^m values of each vector (as qk_fwht / qk_fftbr return it) and x_new = its
 * next n values (raw; transformed in place here), out = the transform of all 2n values:
 *   out = [xt_old + w (.) xt_new, xt_old - w (.) xt_new] / sqrt(2),
 * w_k = 1 (qk_fwht_extend) or exp(-pi i k / n) (qk_fftbr_extend; interleaved complex).
 * xt_old, x_new: (nvec, n); out: (nvec, 2n).  out must not overlap the inputs, nor
 * x_new (transformed in place) xt_old: overlapping arrays return QK_EINVAL. */
QK_API int qk_fwht_extend(uint32_t m, uint64_t nvec, int32_t dtype, const void *xt_old, void *x_new, void *out,
                          qk_stream stream);
QK_API int qk_fftbr_extend(uint32_t m, uint64_t nvec, int32_t dtype, const void *xt_old, void *x_new, void *out,
                           qk_stream stream);

/* qk_fwht with a workspace: the same transform (bit for bit: the same butterflies in the
 * same order), for 2^13 < n <= 2^21 (FP32) or 2^12 < n <= 2^20 (FP64) run either as two
 * launches (low bits on contiguous tiles, then high bits on column tiles) or as ONE
 * persistent launch in which resident CTAs take tiles from a global ticket counter and a
 * vector's column tiles are queued `lag` vectors after its low tiles, so that its
 * first-pass output is still in L2 when read back.  Which one runs, with which lag and
 * CTAs per SM, is the choice qk_fwht_tune recorded for (device, m, dtype, nvec), else the
 * persistent launch with a lag from the grid size; a non-NULL `plan` (host) overrides
 * both.  Other sizes run qk_fwht's transform.
 * ws: (1 + nvec) 32-bit counters, 256-byte aligned (qk_workspace_bytes op 4; reset by the
 * call itself).  A column tile waits for its vector's low tiles with a bounded wait
 * (about 1 s); past it the tile is skipped and QK_STATUS_TIMEOUT is set in `status`
 * (nullable).  Graph-capturable. */
typedef struct {
  int32_t mode;          /* QK_FWHT_TWO_PASS or QK_FWHT_PERSISTENT */
  uint32_t lag;          /* persistent: vectors between low and column tiles (0 = automatic) */
  uint32_t ctas_per_sm;  /* persistent: resident CTAs per SM (0 = the occupancy limit) */
  float ms;              /* tuner: measured milliseconds per transform of the batch */
} qk_fwht_plan;
#define QK_FWHT_TWO_PASS 0
#define QK_FWHT_PERSISTENT 1
QK_API int qk_fwht_ws(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes,
                      const qk_fwht_plan *plan, uint32_t *status, qk_stream stream);

/* qk_fftbr (inverse = 0) or qk_ifftbr (inverse = 1) with a workspace: the same transform,
 * bit for bit, for FP32 and 2^16 <= n <= 2^20 run as ONE persistent launch in which
 * resident CTAs take tiles from a global ticket counter: the contiguous 12-bit tiles and
 * the column tiles of the remaining high bits (FFTBR: in that order; IFFTBR: reversed), a
 * vector's second-pass tiles queued `lag` vectors after its first-pass tiles (0 = from the
 * grid size and n) so that they read the first pass's output back from L2.  Other sizes
 * and FP64 run the transform of qk_fftbr / qk_ifftbr.  ws: (1 + nvec) 32-bit counters,
 * 256-byte aligned (qk_workspace_bytes op 4), reset by the call.  The wait of a
 * second-pass tile is bounded (about 1 s); past it the tile is skipped and
 * QK_STATUS_TIMEOUT set in `status` (nullable).  Graph-capturable. */
QK_API int qk_fftbr_ws(uint32_t m, uint64_t nvec, int32_t dtype, int32_t inverse, void *x, void *ws,
                       size_t ws_bytes, uint32_t lag, uint32_t *status, qk_stream stream);

/* Autotuner for qk_fwht_ws (the paper has no counterpart): times the two-launch form and
 * the persistent launch over CTAs per SM x lag on the caller's buffer x (its contents are
 * overwritten: used as scratch), records the fastest for (current device, m, dtype, nvec)
 * and returns it in *best (nullable).  Synchronises the stream; not capturable. */
QK_API int qk_fwht_tune(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes,
                        qk_fwht_plan *best, qk_stream stream);

/* Test of the persistent launch's bounded wait (no counterpart in the paper): runs only
 * the column tiles of qk_fwht_ws with no low tile published, so that every wait runs
 * out after spin_limit sleeps of ~128 ns (1 .. 2^23); each tile is then skipped (x is
 * left unchanged) and QK_STATUS_TIMEOUT is set in `status` (required). */
QK_API int qk_fwht_wait_selftest(uint32_t m, uint64_t nvec, int32_t dtype, void *x, void *ws, size_t ws_bytes,
                                 uint32_t spin_limit, uint32_t *status, qk_stream stream);

/* Test of the FP64 quotient of the gradient sweeps (no counterpart in the paper): q[i] =
 * a[i] / b[i] as those sweeps form it (two Newton steps on the FP32 reciprocal estimate,
 * then a product; the divide for b outside 2^-100 .. 2^100 in magnitude); a, b, q: n device
 * doubles.  Within 2 ulp of the correctly rounded quotient. */
QK_API int qk_ratio_selftest(const double *a, const double *b, double *q, uint64_t n, qk_stream stream);

/* --------------------------------------------------- higher-order nets --- */

/* Digital interlacing of order alpha (Sec. 4.3, "Digital interlacing for higher-order
 * nets"): from the generator columns Ct (R, alpha d, 32) of an alpha d-dimensional net (for
 * higher-order LMS: the qk_lms_setup output on the alpha d matrices), the d interlaced
 * matrices Chat (R, d, 32) of 64-bit columns, bit 63 - t = digit t, where digit t of matrix j
 * (0-based) is digit floor(t / alpha) of matrix alpha j + (t mod alpha).  The interlaced
 * matrices have 32 alpha digits; the first min(64, 32 alpha) are kept (later digits lie
 * below 2^-64).  alpha in 1..4. */
QK_API int qk_interlace(uint32_t d, uint32_t R, uint32_t alpha, const uint32_t *Ct, uint64_t *Chat,
                        qk_stream stream);

/* A randomized higher-order (interlaced) net: points are 64-digit words, x = X 2^-64. */
typedef struct {
  int32_t order;         /* QK_NATURAL or QK_GRAY */
  uint32_t d;            /* dimensions of the interlaced net */
  uint32_t R;            /* randomizations stored in Chat / D */
  const uint64_t *Chat;  /* (R, d, 32) interlaced columns (qk_interlace output) */
  const uint64_t *D;     /* (R, d) 64-digit digital shifts; NULL means no shift */
} qk_hopointset;

/* Points of a higher-order net, as qk_gen_points: X (nr, n, d) uint64 row-major,
 * X = D (+) XOR_{bit k of g(i)} Chat[:, k] (g(i) = i or its Gray code); i0 + n <= 2^32. */
QK_API int qk_gen_points_ho(const qk_hopointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n,
                            uint64_t *X, qk_stream stream);

/* First Gram column of a product DSI kernel (k->family QK_DSI, order k->alpha 1..4, Sec. 5.3)
 * on the points of a higher-order net, as qk_kernel_col: the Theorem's closed forms at
 * x = Z 2^-64 for the 64-digit difference words Z = X_i (+) X_0 (beta = clz64(Z) + 1; the
 * order-4 digit series over 64 digits).  col: (nr, 2^m) in dtype (QK_F64 / QK_F32) and form.
 * The column feeds qk_eigs, qk_solve, qk_matvec, qk_discrepancy and qk_mll_spectrum
 * unchanged (the Gram matrix of an interlaced net is RSBT). */
QK_API int qk_kernel_col_ho(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m,
                            int32_t dtype, int32_t form, void *col, qk_stream stream);

/* qk_mll for a higher-order net: the MLL pieces and (grad non-NULL) the gradient block of
 * qk_mll, the factors recomputed from the 64-digit words.  lam: (nr, 2^m) from qk_eigs on
 * qk_kernel_col_ho's column (nugget included); y: (nr, nrhs, 2^m) in dtype; out:
 * (nr, nrhs, QK_MLL_NOUT); grad: (nr, nrhs, 2d + 2), nr nrhs <= 65535.  Workspace:
 * qk_workspace_bytes op 3 with (QK_DSI, m, nr, nrhs, dtype, d). */
QK_API int qk_mll_ho(const qk_hopointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m, uint32_t nrhs,
                     int32_t dtype, const double *lam, const void *y, double *out, double *grad, void *ws,
                     size_t ws_bytes, qk_stream stream);

/* The MLL pieces of qk_mll (quadratic form, log det, MLL, posterior mean and variance) from
 * the eigenvalues alone, without the point set (and so without the gradient): for callers
 * that hold only a spectrum.  lam: (nr, 2^m) from qk_eigs;
 * y: (nr, nrhs, 2^m) in dtype; out: (nr, nrhs, QK_MLL_NOUT).  Workspace: qk_workspace_bytes
 * op 3 with d = 0. */
QK_API int qk_mll_spectrum(int32_t family, uint32_t m, uint32_t nr, uint32_t nrhs, int32_t dtype, double zeta,
                           const double *lam, const void *y, double *out, void *ws, size_t ws_bytes,
                           qk_stream stream);

/* ---------------------------------------------------- RQMC integration --- */

/* The test integrands of the numerical experiments (Sec. 6):
 *   QK_F_SIMPLE1   d = 1:  x e^x - 1
 *   QK_F_SIMPLE2   d = 2:  x_2 e^{x_1 x_2} / (e - 2) - 1
 *   QK_F_OAKLEY    d = 2:  g((x - 1/2)/50), g(t) = 5 + t_1 + t_2 + 2 cos t_1 + 2 cos t_2
 *   QK_F_GFUN      any d:  prod_j (|4 x_j - 2| - a_j) / (1 + a_j), a_j = (j - 2)/2
 *   QK_F_GENZ_OSC  any d:  cos(-sum_j c_j x_j), c_j = 4.5 ct_j / sum ct, ct_j = e^{j log(1e-8)/d}
 *   QK_F_GENZ_CP   any d:  (1 + sum_j c_j x_j)^-(d+1), c_j = 0.25 ct_j / sum ct, ct_j = 1/j^2 */
enum qk_integrand_id { QK_F_SIMPLE1 = 0, QK_F_SIMPLE2 = 1, QK_F_OAKLEY = 2, QK_F_GFUN = 3, QK_F_GENZ_OSC = 4,
                       QK_F_GENZ_CP = 5 };

/* y[r][i] = f(x_i) at the points of randomizations r0 .. r0+nr-1, positions i0 .. i0+n-1
 * (the points of qk_gen_points, not materialised), with baker != 0 at the baker-transformed
 * point 1 - 2|x - 1/2| instead (Sec. 4.2: periodises the integrand for lattices, mean
 * unchanged).  y: (nr, n) in dtype (QK_F64 or QK_F32; the arithmetic runs in dtype).
 * The integrand's dimension must match ps->d where it is fixed (QK_EINVAL otherwise). */
QK_API int qk_integrand(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n, int32_t f,
                        int32_t baker, int32_t dtype, void *y, qk_stream stream);

/* RQMC estimate with its Student-t interval (Sec. 3.1, Eq. RQMC): from y (R, n) in dtype
 * (one row of f values per randomization), mu_r = mean_i y[r][i], mu = mean_r mu_r,
 * sigma^2 = sum_r (mu_r - mu)^2 / (R - 1), and the 100(1 - tau)% half width
 * t_{R-1, tau/2} sigma / sqrt(R) (t quantile: qk_student_t_quantile).  out: device doubles
 * (4 + R) = [mu, sigma, half width, t, mu_1 .. mu_R].  R >= 2, 0 < tau < 1. */
QK_API int qk_rqmc(uint32_t R, uint64_t n, int32_t dtype, const void *y, double tau, double *out,
                   qk_stream stream);

/* Host: the p-quantile q of Student's t distribution with df > 0 degrees of freedom
 * (P(T <= q) = p, 0 < p < 1; bisection on the CDF through the regularised incomplete
 * beta function).  *q is a host double. */
QK_API int qk_student_t_quantile(double df, double p, double *q);

/* Squared worst-case error (the generalized kernel discrepancy, Sec. 3.2) of cubature rules
 * on the points of `batch` point sets, for the kernel without nugget: with
 * kappa_i = int K(u, x_i) du = zeta and int int K = zeta (each one-dimensional K_alpha
 * integrates to zero), from the first columns col (batch, n) in dtype and form (QK_COL_P
 * keeps full precision; QK_COL_K1 cancels in k_1/zeta - 1):
 *   out[b][0] = equal weights 1/n:          zeta S / n
 *   out[b][1] = optimal weights K^-1 kappa: zeta - zeta^2 n / lambda_0 = zeta S / (n + S)
 *   out[b][2] = the optimal weight, the same for every point: zeta / lambda_0 = 1 / (n + S)
 * with S = sum_i p_i and lambda_0 = zeta (n + S).  out: (batch, 3) device doubles. */
QK_API int qk_discrepancy(int32_t family, uint32_t m, uint32_t batch, int32_t dtype, int32_t form, const void *col,
                          double zeta, double *out, qk_stream stream);

/* The same for given weights w (batch, nw, n) in dtype:
 *   out[b][q] = zeta - 2 zeta sum_i w_i + w^T K w,  w^T K w = sum_w lambda_w |W_w|^2 / n,
 * W the unnormalised transform of the weights (Sec. 5.4) and lam (batch, n) the eigenvalues
 * of K from qk_eigs with eta = 0.  The difference cancels for near-optimal weights: its
 * absolute error is about eps zeta.  out: (batch, nw) device doubles.  Workspace:
 * qk_workspace_bytes op 5 with (family, m, batch, nrhs = nw, dtype). */
QK_API int qk_discrepancy_weights(int32_t family, uint32_t m, uint32_t batch, uint32_t nw, int32_t dtype,
                                  const double *lam, const void *w, double zeta, double *out, void *ws,
                                  size_t ws_bytes, qk_stream stream);

/* --------------------------------------------------------------- batching --- */

/* One task of a batched schedule: R randomizations of one point set and kernel,
 * n = 2^m points, nrhs right-hand sides per randomization. */
typedef struct {
  qk_pointset ps;
  qk_kernel k;
  uint32_t m;
  uint32_t nrhs;
  double eta;
  const void *y;   /* (R, nrhs, n) in the schedule dtype */
  void *c;         /* (R, nrhs, n) solutions, nullable */
  double *lam;     /* (R, n) eigenvalues out, nullable */
  double *out;     /* (R, nrhs, QK_MLL_NOUT) */
  double *grad;    /* (R, nrhs, 2d+2), nullable */
} qk_task;

/* Workspace for a schedule over host task list `tasks`. */
QK_API int qk_batch_workspace_bytes(const qk_task *tasks, uint32_t ntasks, int32_t dtype,
                             size_t *bytes);

/* Build the device work list of a schedule inside ws (host -> device copy,
 * synchronous with respect to the host).  Must precede qk_batch_run and must
 * be repeated whenever the task list or its pointers change. */
QK_API int qk_batch_plan(const qk_task *tasks, uint32_t ntasks, int32_t dtype, int32_t refine_steps,
                  void *ws, size_t ws_bytes, qk_stream stream);

/* Run a planned schedule: every task's solve, MLL and gradient, in kernel
 * launches only (no host synchronisation, no allocation), so the call can be
 * captured into a CUDA graph. */
QK_API int qk_batch_run(void *ws, size_t ws_bytes, uint32_t *status, qk_stream stream);

/* How qk_batch_run executes a recorded plan.  QK_SCHED_LAUNCHES (the default after
 * qk_batch_plan): per task, a sequence of kernel launches (4 for fused tasks).  Lattice
 * tasks run the column, the eigenvalues and one pass for MLL, gradient and solve (two real
 * vectors per complex FFTBR, one forward transform of y, one inverse transform giving both
 * c and the gradient's back-transformed weights); with QK_F32W the forward transforms and
 * the spectral step are FP64 and the inverse transforms and gradient sweep FP32; a QK_F32
 * schedule with refinement steps keeps a separate refined solve.
 * QK_SCHED_PERSISTENT: ONE launch of resident CTAs for the whole plan; every
 * randomization of every task is a unit whose tiles (column sweep, high-bit transform
 * and epilogue, inverse and gradient sweep, final reduction) are taken in ticket order,
 * a unit's next phase `lag` units (1 or 2; 0 = 1) after its previous one, with bounded
 * waits on per-unit completion counters (QK_STATUS_TIMEOUT if one ever runs out).  The
 * launch takes the plan's DSI nets in the fused size range (2^13 < n <= 2^21 FP32,
 * 2^12 < n <= 2^20 FP64) of the order of the first such task; the other tasks (lattices,
 * other sizes or orders) run after it as their launch sequence on the same stream.
 * QK_EINVAL if no task qualifies.  Uploads the schedule tables into the
 * workspace synchronously: call it outside stream capture; runs are capturable.
 * Results equal the launch sequence's bit for bit.  qk_batch_run_host always uses the
 * launch sequence. */
#define QK_SCHED_LAUNCHES 0
#define QK_SCHED_PERSISTENT 1
QK_API int qk_batch_schedule(void *ws, size_t ws_bytes, int32_t mode, uint32_t lag);

/* Autotuner for a recorded plan (no counterpart in the paper): runs the plan as the
 * launch sequence and, when eligible, as the persistent launch with each lag, times each
 * with CUDA events on `stream` (the plan's outputs are overwritten), and keeps the
 * fastest as the plan's schedule (as qk_batch_schedule would).  Returns the choice and
 * its milliseconds per run (each out-pointer nullable).  Synchronises the stream; not
 * for stream capture. */
QK_API int qk_batch_tune(void *ws, size_t ws_bytes, int32_t *mode, uint32_t *lag, float *ms, qk_stream stream);

/* Run a planned schedule with HOST inputs and outputs (the planned device buffers are
 * the staging area): every task's randomizations go in chunks of at most chunk_r (a half
 * chunk at both ends, so that computing starts after a short first copy and the last copy
 * back is short); chunk k's
 * right-hand sides are copied in on a library stream while chunk k-1 computes, and its
 * results (c, lam, out, grad: those whose host pointer is non-NULL; each needs its device
 * buffer in the plan) are copied back on another library stream while chunk k+1
 * computes.  Chunks compute on `stream`, or, when every task runs fused and two chunks'
 * scratch fits in the workspace in front of the persistent schedule's region, on two
 * library streams in turn, each chunk with its own half of that scratch, so that two
 * chunks' kernels overlap.  io: one qk_host_io per planned task (host pointers, same
 * layouts as the task's device buffers; page-locked memory lets the copies overlap).
 * Returns after enqueueing; `stream` completes after the last copy back.  Not for
 * stream capture.  (The paper has no counterpart: this is the runtime's host path.) */
typedef struct {
  const void *y; /* (R, nrhs, n) in the schedule dtype, required */
  void *c;       /* (R, nrhs, n) or NULL */
  double *lam;   /* (R, n) or NULL */
  double *out;   /* (R, nrhs, QK_MLL_NOUT), required */
  double *grad;  /* (R, nrhs, 2d + 2) or NULL */
} qk_host_io;
QK_API int qk_batch_run_host(void *ws, size_t ws_bytes, const qk_host_io *io, uint32_t chunk_r, uint32_t *status,
                             qk_stream stream);

/* Per-kernel timing of a planned schedule (no paper counterpart; used to report
 * rooflines).  After qk_batch_timing(ws, runs), each of the next `runs` calls of
 * qk_batch_run on that workspace records a CUDA event pair around every kernel it
 * launches, on the launching stream (events are host-side runtime objects; no device
 * memory is allocated).  qk_batch_kernel_ms(ws, idx, ...) waits for the recorded
 * events and returns, for the idx-th distinct kernel name, its launch count and
 * summed device milliseconds; QK_EINVAL once idx runs past the last name.
 * qk_batch_timing(ws, 0) stops recording and forgets the records. */
QK_API int qk_batch_timing(void *ws, uint32_t runs);
QK_API int qk_batch_kernel_ms(void *ws, uint32_t idx, char *name, size_t name_len, uint32_t *launches,
                              double *ms);

/* ------------------------------------------------------------- utilities --- */

/* Workspace bytes needed by qk_eigs / qk_solve / qk_matvec / qk_mll / qk_fwht_ws /
 * qk_discrepancy_weights with these sizes (op: 0 eigs, 1 solve, 2 matvec, 3 mll, 4 fwht_ws
 * with batch = nvec, 5 discrepancy_weights with nrhs = nw). */
QK_API int qk_workspace_bytes(int32_t op, int32_t family, uint32_t m, uint32_t batch, uint32_t nrhs,
                       int32_t dtype, uint32_t d, size_t *bytes);

/* Synchronise `stream`, read the device status word, clear it, and return the
 * corresponding qk_status (QK_OK, QK_ENOTPD or QK_ETIMEOUT). */
QK_API int qk_read_status(uint32_t *status, qk_stream stream);

/* Message of the last failure on this host thread (NUL-terminated, truncated). */
QK_API void qk_last_error(char *buf, size_t len);

/* Number of CUDA kernels this library has launched in this process (all
 * threads, all devices), for accounting launches inside a timed region. */
QK_API uint64_t qk_launch_count(void);

/* Library version as major*10000 + minor*100 + patch. */
QK_API int qk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QK_H */
