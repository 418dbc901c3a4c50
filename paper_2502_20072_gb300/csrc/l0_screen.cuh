// l0_screen.cuh -- declarations of the screening and dimension-loop
// launchers (l0_sis.cu, l0_loop.cu), kept apart from the l0 search's shared
// header.
#pragma once

#include <cuda_runtime.h>

namespace l0 {

// SIS screening (paper Sec. 2.3, Eq. 1): Pearson r of every feature with
// each of R targets, the m largest max_t |r_t| (ties: smaller index) into
// out_idx / out_r (device); err 5 on NaN/Inf, 12 when more than 2^22
// candidates tie at the cut
constexpr int SIS_MAX_TARGETS = 16;
// generated candidates: ops[t](child c1[t], child c2[t]) with the value rules
// (bounds lb <= max |value| <= ub); valid (optional) receives 1 / 0 per
// candidate
struct SisGen {
  long long n_child;          // rows of the children X; a candidate outside: err 14
  const int *ops, *c1, *c2;
  double lb, ub;
  unsigned char *valid;
  // FP32 pre-screen (with prescreen set and valid null): an FP32 copy of the
  // children [n_child][n] and a flag per child (scratch the caller owns)
  float *cf = nullptr;
  unsigned char *csafe = nullptr;
};
size_t sis_scratch_bytes(long long n_feat, int m, long long n, int R);
cudaError_t launch_sis(const double *X, const double *y, int R, long long n, long long n_feat,
                       int m, const int *ex, long long n_ex, int prescreen, void *scratch,
                       int *out_idx, double *out_r, int *err, cudaStream_t st, cudaEvent_t scan0,
                       cudaEvent_t scan1, const SisGen *gen = nullptr);
// dimension loop helpers (l0_loop.cu)
cudaError_t launch_residuals(const double *X, const double *y, long long n, const int *tuples,
                             int d, int R, double *Q, double *out, cudaStream_t st);
cudaError_t launch_gather_rows(const double *X, long long n, const int *rows, int n_rows,
                               double *out, cudaStream_t st);

}  // namespace l0
