// Krylov vector kernels for GMRES (Arnoldi with classical Gram-Schmidt and selective
// re-orthogonalisation). Vectors are complex64 (mixed precision) or complex128; every inner product
// and norm is accumulated in FP64 across threads and blocks. In the complex64 case each thread first
// sums kChunk consecutive products in FP32 before adding them into its FP64 accumulator, which keeps
// the FP64 add rate (far below the FP32 rate on this part) off the critical path.
#include <type_traits>

#include "green.cuh"

namespace ie {

constexpr int kKThreads = 256;
constexpr int kChunk = 8;
constexpr int kMaxBasis = 128;

int krylov_blocks(long n) {
  long g = (n + (long)kKThreads * kChunk - 1) / ((long)kKThreads * kChunk);
  if (g > kRedBlocks) g = kRedBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Block-reduce NQ double2 accumulators and write them to part[q * kRedBlocks + blockIdx.x].
template <int NQ>
__device__ __forceinline__ void block_store(double2 (&acc)[NQ], int nq, double2* part, int slot0) {
  __shared__ double2 red[NQ][kKThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double2 v = warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int w = 0; w < kKThreads / 32; ++w) s = s + red[threadIdx.x][w];
    part[(long)(slot0 + threadIdx.x) * kRedBlocks + blockIdx.x] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kKThreads) k_dots(const C<T>* __restrict__ V, long ld, int nv,
                                                   const C<T>* __restrict__ w, long n, double2* __restrict__ part,
                                                   int with_norm, const int* __restrict__ skip) {
  if (skip && *skip == 0) return;
  const int k0 = blockIdx.y * kDotGroup;
  const int nk = min(kDotGroup, nv - k0);
  const bool do_norm = with_norm && blockIdx.y == 0;
  double2 acc[kDotGroup + 1];
#pragma unroll
  for (int q = 0; q <= kDotGroup; ++q) acc[q] = make_double2(0.0, 0.0);
  const long step = (long)gridDim.x * kKThreads * kChunk;
  for (long base = (long)blockIdx.x * kKThreads * kChunk; base < n; base += step) {
    C<T> a[kDotGroup + 1];
#pragma unroll
    for (int q = 0; q <= kDotGroup; ++q) a[q] = czero<C<T>>();
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const long e = base + i * kKThreads + threadIdx.x;
      if (e < n) {
        const C<T> we = w[e];
#pragma unroll
        for (int q = 0; q < kDotGroup; ++q)
          if (q < nk) {
            const C<T> v = V[(long)(k0 + q) * ld + e];
            a[q].x += v.x * we.x + v.y * we.y;
            a[q].y += v.x * we.y - v.y * we.x;
          }
        if (do_norm) a[kDotGroup].x += we.x * we.x + we.y * we.y;
      }
    }
#pragma unroll
    for (int q = 0; q <= kDotGroup; ++q) acc[q] = acc[q] + to_c64(a[q]);
  }
  // slots k0..k0+nk-1 hold the dots; the norm goes to slot nv (written by group 0 only)
  double2 out[kDotGroup + 1];
#pragma unroll
  for (int q = 0; q < kDotGroup; ++q) out[q] = acc[q];
  out[kDotGroup] = acc[kDotGroup];
  __shared__ double2 red[kDotGroup + 1][kKThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q <= kDotGroup; ++q) {
    double2 v = warp_sum(out[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x <= kDotGroup) {
    const int q = threadIdx.x;
    const bool isnorm = (q == kDotGroup);
    if ((isnorm && do_norm) || (!isnorm && q < nk)) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int w2 = 0; w2 < kKThreads / 32; ++w2) s = s + red[q][w2];
      const int slot = isnorm ? nv : k0 + q;
      part[(long)slot * kRedBlocks + blockIdx.x] = s;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kKThreads) k_update(const C<T>* __restrict__ V, long ld, int nv,
                                                     const double2* __restrict__ h, C<T>* __restrict__ w, long n,
                                                     double2* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip == 0) return;
  __shared__ C<T> hs[kMaxBasis];
  for (int k = threadIdx.x; k < nv; k += kKThreads) hs[k] = to_c(h[k], T());
  __syncthreads();
  double2 acc[1] = {make_double2(0.0, 0.0)};
  const long step = (long)gridDim.x * kKThreads * kChunk;
  for (long base = (long)blockIdx.x * kKThreads * kChunk; base < n; base += step) {
    T a = 0;
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const long e = base + i * kKThreads + threadIdx.x;
      if (e < n) {
        C<T> r = w[e];
        int k = 0;
        for (; k + 4 <= nv; k += 4) {
          const C<T> v0 = V[(long)k * ld + e], v1 = V[(long)(k + 1) * ld + e];
          const C<T> v2 = V[(long)(k + 2) * ld + e], v3 = V[(long)(k + 3) * ld + e];
          r = r - cmul(hs[k], v0) - cmul(hs[k + 1], v1) - cmul(hs[k + 2], v2) - cmul(hs[k + 3], v3);
        }
        for (; k < nv; ++k) r = r - cmul(hs[k], V[(long)k * ld + e]);
        w[e] = r;
        a += r.x * r.x + r.y * r.y;
      }
    }
    acc[0].x += (double)a;
  }
  if (part) block_store<1>(acc, 1, part, nv);
}

template <typename T>
__global__ void __launch_bounds__(kKThreads) k_combine(const C<T>* __restrict__ V, long ld, int nv,
                                                      const double2* __restrict__ y, C<T>* __restrict__ x, long n) {
  __shared__ C<T> ys[kMaxBasis];
  for (int k = threadIdx.x; k < nv; k += kKThreads) ys[k] = to_c(y[k], T());
  __syncthreads();
  for (long e = (long)blockIdx.x * kKThreads + threadIdx.x; e < n; e += (long)gridDim.x * kKThreads) {
    C<T> r = x[e];
    for (int k = 0; k < nv; ++k) r = r + cmul(ys[k], V[(long)k * ld + e]);
    x[e] = r;
  }
}

template <typename T>
__global__ void k_scale(const C<T>* __restrict__ src, C<T>* __restrict__ dst, long n, const double2* __restrict__ nrm2,
                        double host_scale) {
  double s = host_scale;
  if (nrm2) {
    const double v = nrm2->x;
    s = v > 0.0 ? 1.0 / sqrt(v) : 0.0;
  }
  const T st = (T)s;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const C<T> v = src[e];
    dst[e] = mk<T>(st * v.x, st * v.y);
  }
}

template <typename T>
__global__ void __launch_bounds__(kKThreads) k_norm2(const C<T>* __restrict__ v, long n, double2* __restrict__ part,
                                                    const C<T>* __restrict__ b, C<T>* __restrict__ y) {
  // b == nullptr: |v|^2 ; otherwise y = b - y first and |y|^2
  double2 acc[1] = {make_double2(0.0, 0.0)};
  const long step = (long)gridDim.x * kKThreads * kChunk;
  for (long base = (long)blockIdx.x * kKThreads * kChunk; base < n; base += step) {
    T a = 0;
#pragma unroll
    for (int i = 0; i < kChunk; ++i) {
      const long e = base + i * kKThreads + threadIdx.x;
      if (e < n) {
        C<T> r;
        if (b) {
          r = b[e] - y[e];
          y[e] = r;
        } else {
          r = v[e];
        }
        a += r.x * r.x + r.y * r.y;
      }
    }
    acc[0].x += (double)a;
  }
  block_store<1>(acc, 1, part, 0);
}

__global__ void k_reduce(const double2* __restrict__ part, int nblk, double2* __restrict__ out,
                         double2* __restrict__ out2, const int* __restrict__ skip) {
  if (skip && *skip == 0) return;
  const int k = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s = s + part[(long)k * kRedBlocks + b];
  __shared__ double2 red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0.0, 0.0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = t + red[w];
    out[k] = t;
    if (out2) out2[k] = out2[k] + t;
  }
}

__global__ void k_reorth_flag(const double2* nb, const double2* na, double eta2, int* flag) {
  *flag = (na->x < eta2 * nb->x) ? 1 : 0;
}

// ------------------------------------------------------------------ strided c128 / c64 helpers
__global__ void k_c128_to_c64(const double2* __restrict__ src, long scs, float2* __restrict__ dst, long dcs, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    const double2 v = src[c * scs + e];
    dst[c * dcs + e] = make_float2((float)v.x, (float)v.y);
  }
}
__global__ void k_add_c64_to_c128(const float2* __restrict__ src, long scs, double2* __restrict__ dst, long dcs,
                                  long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    dst[c * dcs + e] = dst[c * dcs + e] + to_c64(src[c * scs + e]);
  }
}
__global__ void k_add_c128(const double2* __restrict__ src, long scs, double2* __restrict__ dst, long dcs, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    dst[c * dcs + e] = dst[c * dcs + e] + src[c * scs + e];
  }
}
__global__ void k_copy_c128(const double2* __restrict__ src, long scs, double2* __restrict__ dst, long dcs, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    dst[c * dcs + e] = src[c * scs + e];
  }
}
__global__ void __launch_bounds__(kKThreads) k_norm2_c128(const double2* __restrict__ a, long acs,
                                                         const float2* __restrict__ b, long bcs, long n,
                                                         double2* __restrict__ part) {
  double2 acc[1] = {make_double2(0.0, 0.0)};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    double2 v = a[c * acs + e];
    if (b) v = v + to_c64(b[c * bcs + e]);
    acc[0].x += v.x * v.x + v.y * v.y;
  }
  block_store<1>(acc, 1, part, 0);
}

// ------------------------------------------------------------------ launchers
template <typename T>
cudaError_t Krylov<T>::dots(const C<T>* V, long ld, int nv, const C<T>* w, long n, double2* part, bool with_norm,
                            const int* skip, cudaStream_t s) {
  dim3 grd(krylov_blocks(n), (nv + kDotGroup - 1) / kDotGroup);
  if (nv == 0) grd.y = 1;
  k_dots<T><<<grd, kKThreads, 0, s>>>(V, ld, nv, w, n, part, with_norm ? 1 : 0, skip);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::update(const C<T>* V, long ld, int nv, const double2* h, C<T>* w, long n, double2* part,
                              const int* skip, cudaStream_t s) {
  if (nv > kMaxBasis) return cudaErrorInvalidValue;
  k_update<T><<<krylov_blocks(n), kKThreads, 0, s>>>(V, ld, nv, h, w, n, part, skip);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::combine(const C<T>* V, long ld, int nv, const double2* y, C<T>* x, long n, cudaStream_t s) {
  if (nv > kMaxBasis) return cudaErrorInvalidValue;
  k_combine<T><<<krylov_blocks(n) * kChunk, kKThreads, 0, s>>>(V, ld, nv, y, x, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::scale(const C<T>* src, C<T>* dst, long n, const double* nrm2, double host_scale,
                             cudaStream_t s) {
  k_scale<T><<<krylov_blocks(n) * kChunk, kKThreads, 0, s>>>(src, dst, n, reinterpret_cast<const double2*>(nrm2),
                                                             host_scale);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::norm2(const C<T>* v, long n, double2* part, cudaStream_t s) {
  k_norm2<T><<<krylov_blocks(n), kKThreads, 0, s>>>(v, n, part, nullptr, nullptr);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::rsub(const C<T>* b, C<T>* y, long n, double2* part, cudaStream_t s) {
  k_norm2<T><<<krylov_blocks(n), kKThreads, 0, s>>>(nullptr, n, part, b, y);
  return cudaGetLastError();
}
template struct Krylov<float>;
template struct Krylov<double>;

cudaError_t launch_reduce(const double2* part, int nblk, int nk, double2* out, double2* out2, const int* skip,
                          cudaStream_t s) {
  if (nk <= 0) return cudaSuccess;
  k_reduce<<<nk, 256, 0, s>>>(part, nblk, out, out2, skip);
  return cudaGetLastError();
}
cudaError_t launch_reorth_flag(const double2* nb, const double2* na, double eta2, int* flag, cudaStream_t s) {
  k_reorth_flag<<<1, 1, 0, s>>>(nb, na, eta2, flag);
  return cudaGetLastError();
}
static unsigned egrid(long n) {
  long g = (3 * n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}
cudaError_t launch_c128_to_c64(const double2* src, long scs, float2* dst, long dcs, long n, cudaStream_t s) {
  k_c128_to_c64<<<egrid(n), 256, 0, s>>>(src, scs, dst, dcs, n);
  return cudaGetLastError();
}
cudaError_t launch_add_c64_to_c128(const float2* src, long scs, double2* dst, long dcs, long n, cudaStream_t s) {
  k_add_c64_to_c128<<<egrid(n), 256, 0, s>>>(src, scs, dst, dcs, n);
  return cudaGetLastError();
}
cudaError_t launch_add_c128(const double2* src, long scs, double2* dst, long dcs, long n, cudaStream_t s) {
  k_add_c128<<<egrid(n), 256, 0, s>>>(src, scs, dst, dcs, n);
  return cudaGetLastError();
}
cudaError_t launch_copy_c128(const double2* src, long scs, double2* dst, long dcs, long n, cudaStream_t s) {
  k_copy_c128<<<egrid(n), 256, 0, s>>>(src, scs, dst, dcs, n);
  return cudaGetLastError();
}
cudaError_t launch_norm2_c128(const double2* a, long acs, const float2* b, long bcs, long n, double2* part,
                              cudaStream_t s) {
  k_norm2_c128<<<kRedBlocks, kKThreads, 0, s>>>(a, acs, b, bcs, n, part);
  return cudaGetLastError();
}

}  // namespace ie
