// Declarations of the FP64 setup / receiver launchers (green.cu) and the Krylov vector launchers
// (krylov.cu).
#pragma once
#include "common.cuh"

namespace ie {

constexpr int kMaxRx = 8;  // receivers handled per k_receivers launch

cudaError_t launch_green_tab(double2* out, int comp, int Lx, int Ly, int Lz, int nx, int ny, int nz, double h,
                             double2 k, double sigma0, double2 self, cudaStream_t s);
cudaError_t launch_extract_octant(const double2* full, int Lx, int Ly, int Lz, double scale, double2* o64,
                                  float2* o32, cudaStream_t s);
cudaError_t launch_set_contrast(const double* s6, long N, double sigma0, double* d64, float* d32, int* bad,
                                cudaStream_t s);
cudaError_t launch_incident_E(double2* E0, int nx, int ny, int nz, const double* origin, double h, const double* pos,
                              const double* m, double2 k, double omega_mu0, cudaStream_t s);
int receivers_partials_blocks(long N);
cudaError_t launch_receivers(const double2* E, long e_cs, const double* ds, long N, int nx, int ny, const double* origin,
                             double h, const double* rx_dev, int n_rx, double2 k, double2* part, const double* src_pos,
                             const double* m, double2* H, cudaStream_t s);

// ------------------------------------------------------------------ Krylov vector operations
// Vectors are n complex entries (float2 or double2); a basis is nv vectors at stride ld.
constexpr int kDotGroup = 8;    // basis vectors per dot-product block row
constexpr int kRedBlocks = 608;  // upper bound on partial-sum blocks (4 per SM)

template <typename T> struct Krylov {
  // part[k * kRedBlocks + b] = sum over block b of conj(V_k) w   (k < nv);  part[nv*kRedBlocks + b] = |w|^2
  static cudaError_t dots(const C<T>* V, long ld, int nv, const C<T>* w, long n, double2* part, bool with_norm,
                          const int* skip, cudaStream_t s);
  // w -= sum_k h_k V_k; optional |w|^2 partials into part (as .x)
  static cudaError_t update(const C<T>* V, long ld, int nv, const double2* h, C<T>* w, long n, double2* part,
                            const int* skip, cudaStream_t s);
  // x += sum_k y_k V_k
  static cudaError_t combine(const C<T>* V, long ld, int nv, const double2* y, C<T>* x, long n, cudaStream_t s);
  // dst = src * scale, scale = 1/sqrt(*nrm2) (0 if *nrm2 == 0) or a host value when nrm2 == nullptr
  static cudaError_t scale(const C<T>* src, C<T>* dst, long n, const double* nrm2, double host_scale, cudaStream_t s);
  // partial |v|^2
  static cudaError_t norm2(const C<T>* v, long n, double2* part, cudaStream_t s);
  // y = b - y  (used for the true residual b - A x with A x already in y); |y|^2 partials
  static cudaError_t rsub(const C<T>* b, C<T>* y, long n, double2* part, cudaStream_t s);
};
int krylov_blocks(long n);
// out[k] = sum_b part[k*kRedBlocks + b] for k < nk (nblk partials per row); if out2, also out2[k] += out[k].
// Skipped entirely when skip != nullptr and *skip == 0.
cudaError_t launch_reduce(const double2* part, int nblk, int nk, double2* out, double2* out2, const int* skip,
                          cudaStream_t s);
// flag = (nrm2_after < eta^2 * nrm2_before): reorthogonalisation needed
cudaError_t launch_reorth_flag(const double2* nrm_before, const double2* nrm_after, double eta2, int* flag,
                               cudaStream_t s);

// c128 <-> c64 helpers on strided 3-component fields (slab of a whole-domain field)
cudaError_t launch_c128_to_c64(const double2* src, long src_cs, float2* dst, long dst_cs, long n, cudaStream_t s);
cudaError_t launch_add_c64_to_c128(const float2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
cudaError_t launch_add_c128(const double2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
cudaError_t launch_copy_c128(const double2* src, long src_cs, double2* dst, long dst_cs, long n, cudaStream_t s);
// partial sums of |a + b|^2 (b may be null) over a 3-component strided field (FP64 inputs or f32 b)
cudaError_t launch_norm2_c128(const double2* a, long a_cs, const float2* b, long b_cs, long n, double2* part,
                              cudaStream_t s);

}  // namespace ie
