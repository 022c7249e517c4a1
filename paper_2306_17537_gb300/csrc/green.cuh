// Declarations of the FP64 setup / receiver launchers (green.cu) and the Krylov vector launchers
// (krylov.cu).
#pragma once
#include <cstddef>
#include "common.cuh"

namespace ie {

constexpr int kMaxRx = 8;  // receivers handled per k_receivers launch

cudaError_t launch_green_tab(double2* out, int comp, int Lx, int Ly, int Lz, int nx, int ny, int nz, double h,
                             double2 k, double sigma0, double2 self, cudaStream_t s);
// octant of the scaled spectrum in complex128, complex64 and double-float (odf: [n] x 16 bytes)
cudaError_t launch_extract_octant(const double2* full, int Lx, int Ly, int Lz, double scale, double2* o64,
                                  float2* o32, void* odf, cudaStream_t s);
// act[z] = 1 when plane z (nxy cells) has any non-zero contrast component (d64 [6][N]).
cudaError_t launch_plane_active(const double* d64, long N, long nxy, int nz, int* act, cudaStream_t s);
// Contraction form: M = 2 sigma0 (dsigma + 2 sigma0 I)^-1 and K = dsigma M from the FP64 contrast.
cudaError_t launch_contract_tensors(const double* d64, long N, double sigma0, double* K64, double* M64, float* K32,
                                    float* M32, cudaStream_t s);
// x := M x in place (M symmetric [6][...] at stride m_cs; x [3][n] at stride cs).
cudaError_t launch_apply_sym6(const float* M, long m_cs, float2* x, long cs, long n, cudaStream_t s);
cudaError_t launch_apply_sym6(const double* M, long m_cs, double2* x, long cs, long n, cudaStream_t s);
cudaError_t launch_set_contrast(const double* s6, long N, double sigma0, double* d64, float* d32, int* bad,
                                cudaStream_t s);
cudaError_t launch_incident_E(double2* E0, int nx, int ny, int nz, const double* origin, double h, const double* pos,
                              const double* m, double2 k, double omega_mu0, cudaStream_t s);
int receivers_partials_blocks(long N);
cudaError_t launch_receivers(const double2* E, long e_cs, const double* ds, long N, int nx, int ny, const double* origin,
                             double h, const double* rx_dev, int n_rx, double2 k, double2* part, const double* src_pos,
                             const double* m, double2* H, cudaStream_t s);

// ------------------------------------------------------------------ Krylov vector operations
// Vectors are n complex entries (float2 or double2), 16-byte aligned; a basis is nv vectors at
// stride ld (ld even). Every reduction finishes inside its kernel (last block) and writes FP64
// results to device memory; RedScratch holds the per-block partials and the arrival counters
// (zero-initialised once, reset by the kernels).
constexpr int kDotGroup = 8;     // basis vectors per dot-product block row
constexpr int kRedBlocks = 608;  // upper bound on reduction blocks (4 per SM)
constexpr int kRedSlots = 136;   // partial-sum rows (basis up to 127 vectors + norm)
constexpr int kCounterUpdate = 16, kCounterNorm = 17, kCounters = 32;
struct RedScratch {
  double2* part;       // [kRedSlots][kRedBlocks]
  unsigned* counters;  // [kCounters], zero
};

template <typename T> struct Krylov {
  // out[k] = V_k^H w (k < nv) and, with_norm, out[nv] = |w|^2; acc[k] += out[k] when acc != null.
  // Does nothing when skip != null and *skip == 0.
  static cudaError_t dots(const C<T>* V, long ld, int nv, const C<T>* w, long n, bool with_norm, double2* out,
                          double2* acc, const int* skip, const RedScratch& sc, cudaStream_t s);
  // w -= sum_k h_k V_k, *out_norm = |w|^2; with flag: *flag = (|w|^2 < eta2 * ref->x). skip as above.
  static cudaError_t update(const C<T>* V, long ld, int nv, const double2* h, C<T>* w, long n, double2* out_norm,
                            const double2* ref, double eta2, int* flag, const int* skip, const RedScratch& sc,
                            cudaStream_t s);
  // x += sum_k y_k V_k (k < nv, or k < *nv_dev when nv_dev is not null; nv is then the upper bound)
  static cudaError_t combine(const C<T>* V, long ld, int nv, const double2* y, C<T>* x, long n, cudaStream_t s,
                             const int* nv_dev = nullptr);
  // dst = src / sqrt(nrm2->x) (0 if the norm is 0), or dst = src * host_scale when nrm2 is null
  static cudaError_t scale(const C<T>* src, C<T>* dst, long n, const double2* nrm2, double host_scale, cudaStream_t s);
  // *out = |v|^2
  static cudaError_t norm2(const C<T>* v, long n, double2* out, const RedScratch& sc, cudaStream_t s);
  // y = b - y, *out = |y|^2  (true residual b - A x with A x already in y)
  static cudaError_t rsub(const C<T>* b, C<T>* y, long n, double2* out, const RedScratch& sc, cudaStream_t s);
};
int krylov_blocks(long n);

// ---------------------------------------------------------------- GMRES driven from the device
// State of one restarted GMRES solve whose Givens rotations, stopping tests and restarts run on the
// device (one CUDA graph per solve; see gm_* launchers). FP64 throughout.
constexpr int kGmMaxM = 128;     // restart length limit (the host path allows 127)
constexpr int kGmMaxCycles = 512;  // restart cycles whose lengths are recorded for the accounting
struct GmState {
  int j;        // Arnoldi steps done in the current cycle
  int iters;    // Arnoldi steps in total
  int cycles;   // restart cycles finished
  int status;   // 0 running, 1 converged, 2 iteration limit or breakdown with residual > tol, 3 non-finite
  int jd;       // steps of the cycle being combined (back-substitution length)
  int reorth;   // Arnoldi steps that took the second Gram-Schmidt pass
  int max_it, m;
  double tol, bnorm, beta, rel, est, spare;
  double2 cs[kGmMaxM], sn[kGmMaxM], g[kGmMaxM + 1], y[kGmMaxM];
  double2 H[(kGmMaxM + 1) * kGmMaxM];  // rotated Hessenberg, (i, j) at i * kGmMaxM + j
  int cyc_len[kGmMaxCycles];
};
// The scalar head of GmState, as read back by the host.
struct GmHead {
  int j, iters, cycles, status, jd, reorth, max_it, m;
  double tol, bnorm, beta, rel, est, spare;
};
static_assert(sizeof(GmHead) == offsetof(GmState, cs), "GmHead must mirror the head of GmState");
// bnorm from nrm2 (|b|^2); opens the solve (outer condition = bnorm > 0)
cudaError_t gm_init(GmState* st, const double2* nrm2, cudaGraphConditionalHandle outer, cudaStream_t s);
// Conditions of the m Arnoldi-step IF nodes of one cycle (a handle serves exactly one node).
struct GmSteps {
  cudaGraphConditionalHandle h[kGmMaxM];
  int m;
};
// starts a restart cycle: j = 0, g = (beta, 0, ...); step 0 enabled, steps 1..m-1 disabled
cudaError_t gm_cycle(GmState* st, const GmSteps& steps, cudaStream_t s);
// Arnoldi step j: Hessenberg column from h[0..j] and |w|^2 (nrm2), rotations, residual estimate;
// enables step j+1 (next, if j+1 < m) unless the estimate meets tol, the step broke down or the
// iteration limit is reached
cudaError_t gm_step(GmState* st, int j, const double2* h, const double2* nrm2, const int* reorth_flag,
                    cudaGraphConditionalHandle next, bool has_next, cudaStream_t s);
// back substitution of the current cycle into y (written as double2 to y_out) and st->jd
cudaError_t gm_solve(GmState* st, double2* y_out, cudaStream_t s);
// true residual |b - A x|^2 in nrm2: convergence / limit test, outer condition
cudaError_t gm_restart(GmState* st, const double2* nrm2, cudaGraphConditionalHandle outer, cudaStream_t s);

// c128 <-> c64 helpers on strided 3-component fields (slab of a whole-domain field)
cudaError_t launch_c128_to_c64(const double2* src, long src_cs, float2* dst, long dst_cs, long n, cudaStream_t s);
cudaError_t launch_add_c64_to_c128(const float2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
cudaError_t launch_add_c128(const double2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
// acc += a - b (contiguous complex64 vectors of n3 elements)
cudaError_t launch_add_diff_c64(float2* acc, const float2* a, const float2* b, long n3, cudaStream_t s);
cudaError_t launch_copy_c128(const double2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
// *out = |a + b|^2 over a 3-component strided field (b optional, complex64)
cudaError_t launch_norm2_c128(const double2* a, long a_cs, const float2* b, long b_cs, long n, double2* out,
                              const RedScratch& sc, cudaStream_t s);

}  // namespace ie
