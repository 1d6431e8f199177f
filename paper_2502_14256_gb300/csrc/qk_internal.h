// Host-side launchers shared between the libqk translation units.
#pragma once

#include <vector>

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qk.h"

namespace qk {

// Optional per-launch event recorder (qk_batch_timing); begin/end bracket one launch.
struct LaunchTimer {
  virtual void begin(const char *name, cudaStream_t st) = 0;
  virtual void end(cudaStream_t st) = 0;
  virtual ~LaunchTimer() {}
};

// Point-set description resolved for one randomization range.
struct ColJob {
  int32_t kind, order;
  uint32_t d, m;
  const uint32_t *Ct;   // nets: (R, d, 32), already offset to randomization r0
  const uint32_t *g;    // lattices
  const double *w;      // (d) weights
  double zeta;
  int32_t family, alpha;
  uint32_t nr;          // randomizations in this job
  uint64_t i0 = 0;      // first point position (kernel columns of a later block of points)
  const uint64_t *Chat = nullptr;  // higher-order nets (kind kHONet): (R, d, 32) 64-digit columns
};
constexpr int32_t kHONet = 2;  // ColJob kind of an interlaced net (qk_honet.cu)
// Gradient partial sums of a higher-order net job (same layout as launch_grad_partials).
int launch_grad_partials_ho(const ColJob &job, uint32_t nrhs, int32_t dtype, const void *u, double *partial,
                            cudaStream_t st);

// Argument checks of the entry points (qk_api.cu): QK_OK or the error code, message set.
int check_pointset(const qk_pointset *ps, uint32_t r0, uint32_t nr);
int check_kernel(const qk_kernel *k, const qk_pointset *ps);
int check_ws(const void *ws, size_t have, size_t need);

// The job of randomizations r0 .. r0+nr-1 of a (validated) point set and kernel (qk_api.cu).
ColJob make_job(const qk_pointset *ps, const qk_kernel *k, uint32_t r0, uint32_t nr, uint32_t m);

// First column (form QK_COL_K1 / QK_COL_P) of nr randomizations: out (nr, n).
int launch_kernel_col(const ColJob &job, int32_t dtype, int32_t form, void *out, cudaStream_t st);

// Gradient partial sums.  u: (nr * nrhs, n) in dtype (vector v belongs to
// randomization v / nrhs); with `pairs`, u is the pair layout of the lattice transforms
// instead: vector v is the real (v even) or imaginary (v odd) part of complex vector v / 2.
// pcol (nullable): the job's first column in p form, FP64 (nr, n), read instead of a
// second column sweep.  partial: (nr * nrhs, blocks, 2d) doubles with
// blocks = grad_blocks(m): [0, d) sum_i u_i dk1_i/dc_j, [d, 2d) sum_i dk1_i/dc_j.
int launch_grad_partials(const ColJob &job, uint32_t nrhs, int32_t dtype, const void *u,
                         double *partial, cudaStream_t st, bool pairs = false, const double *pcol = nullptr);
uint32_t grad_blocks(uint32_t m);

int launch_gen_points(const qk_pointset *ps, uint32_t r0, uint32_t nr, uint64_t i0, uint64_t n,
                      uint32_t *X, cudaStream_t st);
int launch_lms(uint32_t d, uint32_t R, const uint32_t *C, const uint32_t *S, uint32_t *Ct,
               cudaStream_t st);

bool fused_supported(const qk_task &t, int dtype);
bool tiled_wht_supported(uint32_t m, int dtype);
int tiled_wht(void *x, uint32_t m, uint64_t nvec, int dtype, double scale, cudaStream_t st,
              size_t chunk_bytes = ~(size_t)0);
// Persistent single-launch batched WHT (qk_fused.cu) and its tuner (qk_tune.cu).
constexpr uint32_t kSpinLimit = 1u << 23;  // ~1 s of 128 ns sleeps
size_t persist_wht_ws_bytes(uint64_t nvec);
// Persistent FP32 FFTBR (kind 1) / IFFTBR (kind 2) of n = 2^m, 16 <= m <= 20, in one launch
// (qk_transform.cuh k_fft_persist); ctr: (1 + nvec) counters; lag 0 = automatic.
bool persist_fft_supported(uint32_t m, int dtype);
int persist_fft(int kind, void *x, uint32_t m, uint64_t nvec, double scale, uint32_t *ctr, uint32_t *status,
                uint32_t lag, cudaStream_t st, uint32_t spin_limit = kSpinLimit);
int persist_wht_max_ctas_per_sm(int dtype);
uint32_t persist_wht_default_lag(uint32_t m, uint64_t nvec, int dtype, uint32_t ctas);
int persist_wht(void *x, uint32_t m, uint64_t nvec, int dtype, double scale, void *ws, uint32_t *status,
                cudaStream_t st, uint32_t lag, uint32_t ctas_per_sm, uint32_t spin_limit = kSpinLimit,
                bool columns_only = false);
size_t fused_ws_bytes(const qk_task &t, int dtype, int refine);

// Persistent whole-pipeline schedule (qk_fused.cu): one launch for every randomization of
// every task (all fused DSI nets of one order).
struct PersistState {
  bool ok = false;
  void *units = nullptr, *steps = nullptr, *ctr = nullptr;
  size_t ctr_bytes = 0;
  uint32_t U = 0, S = 0, lag = 0, nslot = 0, dmax = 0;
  int dtype = 0, refine = 0, alpha = 0;
};
bool persist_eligible(const std::vector<qk_task> &tasks, int dtype);
size_t persist_ws_bytes(const std::vector<qk_task> &tasks, int dtype, int refine, uint32_t lag);
int persist_setup(const std::vector<qk_task> &tasks, int dtype, int refine, uint32_t lag, void *region,
                  size_t bytes, PersistState &out);
int persist_run(const PersistState &p, uint32_t *status, cudaStream_t st, LaunchTimer *tm,
                uint32_t spin_limit = kSpinLimit);
int run_fused(const qk_task &t, const ColJob &job, int dtype, int refine, void *ws, uint32_t *status,
              cudaStream_t st, LaunchTimer *tm = nullptr);
}  // namespace qk

namespace qk {
size_t ws_eigs(int family, uint32_t m, uint32_t batch, int dtype);
size_t ws_solve(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype);
size_t ws_matvec(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype);
size_t ws_mll(int family, uint32_t m, uint32_t nr, uint32_t nrhs, int dtype, uint32_t d);
size_t elem_bytes(int family, int dtype);
int op_eigs(int family, uint32_t m, uint32_t batch, int dtype, int form, const void *col, double zeta, double eta,
            double *lam, void *ws, uint32_t *status, cudaStream_t st);
int op_solve(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype, const double *lam, const void *y,
             void *c, int refine, void *ws, cudaStream_t st);
int op_matvec(int family, uint32_t m, uint32_t batch, uint32_t nrhs, int dtype, const double *lam, const void *y,
              void *u, void *ws, cudaStream_t st);
int op_transform(int kind, uint32_t m, uint64_t nvec, int dtype, void *x, cudaStream_t st);
int op_forward_real(int family, uint32_t m, uint64_t nvec, int dtype, const void *in, void *X, cudaStream_t st);
size_t ws_discrepancy(int family, uint32_t m, uint32_t batch, uint32_t nw, int dtype);
int op_eigs_extend(int family, uint32_t m, uint32_t batch, int dtype, int form, const void *col_new, double zeta,
                   double eta, const double *lam_old, double *lam, void *ws, uint32_t *status, cudaStream_t st);
int op_transform_extend(int kind, uint32_t m, uint64_t nvec, int dtype, const void *xt_old, void *x_new, void *out,
                        cudaStream_t st);
// Lattice tasks: MLL, gradient (grad may be null) and solve (c may be null) in one pass on
// pairs of vectors; workspace ws_mll_si(..., c != null).
size_t ws_mll_si(uint32_t m, uint32_t nr, uint32_t nrhs, int dtype, uint32_t d, bool with_c);
int op_mll_solve_si(const ColJob &job, uint32_t nrhs, int dtype, const double *lam, const void *y, double *out,
                    double *grad, void *c, void *ws, cudaStream_t st, const double *pcol = nullptr);
int op_mll(const ColJob &job, uint32_t nrhs, int dtype, const double *lam, const void *y, double *out, double *grad,
           void *ws, cudaStream_t st);
}  // namespace qk
