// Krylov vector kernels for GMRES: Arnoldi by classical Gram-Schmidt with a second pass on demand,
// basis combination, norms.
//
// Vectors are complex64 (mixed precision) or complex128, 16-byte aligned, read as 16-byte packets
// (two complex64 or one complex128 values). Every inner product and norm is reduced in FP64 across
// threads and blocks. Within a thread the complex64 products (a few dozen at most, see krylov_blocks)
// are summed in FP32, across the lanes of a warp in double-float, and the FP64 pipe (a small
// fraction of the FP32 rate on this part) is only used once per warp.
// Each reduction finishes in the last block to arrive (partials summed in a fixed order, so the
// result is deterministic); no separate reduction launch is needed.
#include <algorithm>

#include "green.cuh"

namespace ie {

constexpr int kKThreads = 256;
constexpr int kMaxBasis = 128;

// Blocks for an n-element Krylov kernel: at least 4 packets per thread before the grid reaches
// kRedBlocks, so small sub-domains do not pay for hundreds of partial sums.
int krylov_blocks(long n) {
  long g = (n / 2 + 4L * kKThreads - 1) / (4L * kKThreads);
  if (g > kRedBlocks) g = kRedBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------------ packets and accumulators
template <typename T> struct Pk;
template <> struct Pk<float> {
  using P = float4;
  static constexpr int CPP = 2;
  __device__ __forceinline__ static float2 get(const P& p, int j) { return j ? make_float2(p.z, p.w) : make_float2(p.x, p.y); }
  __device__ __forceinline__ static P make(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
};
template <> struct Pk<double> {
  using P = double2;
  static constexpr int CPP = 1;
  __device__ __forceinline__ static double2 get(const P& p, int) { return p; }
  __device__ __forceinline__ static P make(double2 a, double2) { return a; }
};

template <typename T> struct Acc;  // per-thread complex accumulator
// FP32 per thread: a thread sums at most a few dozen products (the grids are sized to keep it so:
// krylov_blocks), so its rounding stays at a few units of FP32 epsilon relative to the partial sum;
// the sums across threads, where the count grows with n, are carried in double-float and FP64.
template <> struct Acc<float> {
  float2 s = make_float2(0.f, 0.f);
  __device__ __forceinline__ void add(float2 x) {
    s.x += x.x;
    s.y += x.y;
  }
  // Sum over the warp in double-float (FP32 pipes), converted to FP64 once.
  __device__ __forceinline__ double2 warp_total() const {
    df re(s.x, 0.f), im(s.y, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const df r2(__shfl_down_sync(0xffffffffu, re.hi, o), __shfl_down_sync(0xffffffffu, re.lo, o));
      const df i2(__shfl_down_sync(0xffffffffu, im.hi, o), __shfl_down_sync(0xffffffffu, im.lo, o));
      re = re + r2;
      im = im + i2;
    }
    return make_double2(to_double(re), to_double(im));
  }
};
template <> struct Acc<double> {
  double2 s = make_double2(0.0, 0.0);
  __device__ __forceinline__ void add(double2 x) { s = s + x; }
  __device__ __forceinline__ double2 warp_total() const {
    double2 v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_down_sync(0xffffffffu, v.x, o);
      v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
  }
};

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Sum the warp totals over the block in FP64 (lane 0 of each warp holds one); result in thread 0.
__device__ __forceinline__ double2 block_sum_warps(double2 wt, double2* red /* [kKThreads/32] shared */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = wt;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int w = 0; w < kKThreads / 32; ++w) s = s + red[w];
  return s;
}
template <typename T> __device__ __forceinline__ double2 block_sum(const Acc<T>& a, double2* red) {
  return block_sum_warps(a.warp_total(), red);
}
// Sum one FP64 value per thread over the block; result in thread 0.
__device__ __forceinline__ double2 block_sum(double2 v, double2* red) { return block_sum_warps(warp_sum(v), red); }

// Last-block detection after this block has written its partials.
__device__ __forceinline__ bool arrive_last(unsigned* counter, unsigned nblocks) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == nblocks - 1);
  __syncthreads();
  return last;
}

// Fixed-order sum of the partials of one slot by the whole block; result in thread 0.
__device__ __forceinline__ double2 sum_partials(const double2* part, int nblk, double2* red) {
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += kKThreads) s = s + __ldcg(part + b);
  return block_sum(s, red);
}
// Fixed-order sum of the partials of one slot by one warp; result in lane 0.
__device__ __forceinline__ double2 warp_sum_partials(const double2* part, int nblk) {
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x & 31; b < nblk; b += 32) s = s + __ldcg(part + b);
  return warp_sum(s);
}

// ------------------------------------------------------------------ inner products V^H w (+ |w|^2)
template <typename T>
__global__ void __launch_bounds__(kKThreads) k_dots(const C<T>* __restrict__ V, long ld, int nv,
                                                   const C<T>* __restrict__ w, long n, int with_norm,
                                                   double2* __restrict__ part, unsigned* __restrict__ counters,
                                                   double2* __restrict__ out, double2* __restrict__ acc,
                                                   const int* __restrict__ skip) {
  if (skip && *skip == 0) return;
  using K = Pk<T>;
  constexpr int G = kDotGroup, CPP = K::CPP;
  __shared__ double2 red[kKThreads / 32];
  const int g = blockIdx.y, k0 = g * G, nk = min(G, nv - k0);
  const bool dn = with_norm && g == 0;
  Acc<T> a[G];
  Acc<T> an;
  const long np = n / CPP;
  const typename K::P* wp = reinterpret_cast<const typename K::P*>(w);
  for (long p = (long)blockIdx.x * kKThreads + threadIdx.x; p < np; p += (long)gridDim.x * kKThreads) {
    const typename K::P wv = __ldcs(wp + p);
    typename K::P vv[G];
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (q < nk) vv[q] = __ldcs(reinterpret_cast<const typename K::P*>(V + (long)(k0 + q) * ld) + p);
#pragma unroll
    for (int q = 0; q < G; ++q)
      if (q < nk) {
        C<T> t = czero<C<T>>();
#pragma unroll
        for (int j = 0; j < CPP; ++j) {
          const C<T> v = K::get(vv[q], j), x = K::get(wv, j);
          t.x += v.x * x.x + v.y * x.y;
          t.y += v.x * x.y - v.y * x.x;
        }
        a[q].add(t);
      }
    if (dn) {
      T s = 0;
#pragma unroll
      for (int j = 0; j < CPP; ++j) {
        const C<T> x = K::get(wv, j);
        s += x.x * x.x + x.y * x.y;
      }
      an.add(mk<T>(s, 0));
    }
  }
  if (CPP == 2 && (n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {  // odd tail element
    const C<T> x = w[n - 1];
    for (int q = 0; q < nk; ++q) {
      const C<T> v = V[(long)(k0 + q) * ld + n - 1];
      a[q].add(mk<T>(v.x * x.x + v.y * x.y, v.x * x.y - v.y * x.x));
    }
    if (dn) an.add(mk<T>(x.x * x.x + x.y * x.y, 0));
  }
#pragma unroll
  for (int q = 0; q < G; ++q) {
    if (q < nk) {
      const double2 s = block_sum(a[q], red);
      if (threadIdx.x == 0) part[(long)(k0 + q) * kRedBlocks + blockIdx.x] = s;
    }
  }
  if (dn) {
    const double2 s = block_sum(an, red);
    if (threadIdx.x == 0) part[(long)nv * kRedBlocks + blockIdx.x] = s;
  }
  if (!arrive_last(counters + g, gridDim.x)) return;
  // the group's slots (and the norm) in parallel, one warp per slot
  const int nslots = nk + (dn ? 1 : 0);
  for (int q = threadIdx.x >> 5; q < nslots; q += kKThreads / 32) {
    const int slot = (q < nk) ? k0 + q : nv;
    const double2 s = warp_sum_partials(part + (long)slot * kRedBlocks, gridDim.x);
    if ((threadIdx.x & 31) == 0) {
      out[slot] = s;
      if (acc && slot < nv) acc[slot] = acc[slot] + s;
    }
  }
  if (threadIdx.x == 0) counters[g] = 0u;
}

// ------------------------------------------------------------------ w -= sum_k h_k V_k ; |w|^2
template <typename T>
__global__ void __launch_bounds__(kKThreads) k_update(const C<T>* __restrict__ V, long ld, int nv,
                                                     const double2* __restrict__ h, C<T>* __restrict__ w, long n,
                                                     double2* __restrict__ part, unsigned* __restrict__ counter,
                                                     double2* __restrict__ out_norm, const double2* __restrict__ ref,
                                                     double eta2, int* __restrict__ flag, const int* __restrict__ skip) {
  if (skip && *skip == 0) return;
  using K = Pk<T>;
  constexpr int CPP = K::CPP;
  __shared__ C<T> hs[kMaxBasis];
  __shared__ double2 red[kKThreads / 32];
  for (int k = threadIdx.x; k < nv; k += kKThreads) hs[k] = to_c(h[k], T());
  __syncthreads();
  Acc<T> an;
  const long np = n / CPP;
  typename K::P* wp = reinterpret_cast<typename K::P*>(w);
  for (long p = (long)blockIdx.x * kKThreads + threadIdx.x; p < np; p += (long)gridDim.x * kKThreads) {
    const typename K::P wv = wp[p];
    C<T> r[CPP];
#pragma unroll
    for (int j = 0; j < CPP; ++j) r[j] = K::get(wv, j);
    int k = 0;
    for (; k + 4 <= nv; k += 4) {
      typename K::P v4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v4[u] = __ldcs(reinterpret_cast<const typename K::P*>(V + (long)(k + u) * ld) + p);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < CPP; ++j) r[j] = r[j] - cmul(hs[k + u], K::get(v4[u], j));
    }
    for (; k < nv; ++k) {
      const typename K::P v1 = __ldcs(reinterpret_cast<const typename K::P*>(V + (long)k * ld) + p);
#pragma unroll
      for (int j = 0; j < CPP; ++j) r[j] = r[j] - cmul(hs[k], K::get(v1, j));
    }
    wp[p] = K::make(r[0], r[CPP - 1]);
    T s = 0;
#pragma unroll
    for (int j = 0; j < CPP; ++j) s += r[j].x * r[j].x + r[j].y * r[j].y;
    an.add(mk<T>(s, 0));
  }
  if (CPP == 2 && (n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    C<T> r = w[n - 1];
    for (int k = 0; k < nv; ++k) r = r - cmul(hs[k], V[(long)k * ld + n - 1]);
    w[n - 1] = r;
    an.add(mk<T>(r.x * r.x + r.y * r.y, 0));
  }
  const double2 s = block_sum(an, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!arrive_last(counter, gridDim.x)) return;
  const double2 tot = sum_partials(part, gridDim.x, red);
  if (threadIdx.x == 0) {
    *out_norm = tot;
    if (flag) *flag = (tot.x < eta2 * ref->x) ? 1 : 0;
    *counter = 0u;
  }
}

// ------------------------------------------------------------------ x += sum_k y_k V_k
template <typename T>
__global__ void __launch_bounds__(kKThreads) k_combine(const C<T>* __restrict__ V, long ld, int nv,
                                                      const double2* __restrict__ y, C<T>* __restrict__ x, long n,
                                                      const int* __restrict__ nv_dev) {
  __shared__ C<T> ys[kMaxBasis];
  if (nv_dev) nv = min(nv, *nv_dev);
  for (int k = threadIdx.x; k < nv; k += kKThreads) ys[k] = to_c(y[k], T());
  __syncthreads();
  for (long e = (long)blockIdx.x * kKThreads + threadIdx.x; e < n; e += (long)gridDim.x * kKThreads) {
    C<T> r = x[e];
    for (int k = 0; k < nv; ++k) r = r + cmul(ys[k], V[(long)k * ld + e]);
    x[e] = r;
  }
}

// dst = src * s, s = 1/sqrt(nrm2->x) (0 when the norm is 0) or host_scale when nrm2 is null
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

// out = |v|^2, or (b != null) y = b - y and out = |y|^2
template <typename T>
__global__ void __launch_bounds__(kKThreads) k_norm2(const C<T>* __restrict__ v, long n, const C<T>* __restrict__ b,
                                                    C<T>* __restrict__ y, double2* __restrict__ part,
                                                    unsigned* __restrict__ counter, double2* __restrict__ out) {
  __shared__ double2 red[kKThreads / 32];
  Acc<T> an;
  for (long e = (long)blockIdx.x * kKThreads + threadIdx.x; e < n; e += (long)gridDim.x * kKThreads) {
    C<T> r;
    if (b) {
      r = b[e] - y[e];
      y[e] = r;
    } else {
      r = v[e];
    }
    an.add(mk<T>(r.x * r.x + r.y * r.y, 0));
  }
  const double2 s = block_sum(an, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!arrive_last(counter, gridDim.x)) return;
  const double2 tot = sum_partials(part, gridDim.x, red);
  if (threadIdx.x == 0) {
    *out = tot;
    *counter = 0u;
  }
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
// acc += a - b on block-local complex64 vectors of 3n elements
__global__ void k_add_diff_c64(float2* __restrict__ acc, const float2* __restrict__ a, const float2* __restrict__ b,
                               long n3) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n3; i += (long)gridDim.x * blockDim.x)
    acc[i] = acc[i] + (a[i] - b[i]);
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
// out = |a + b|^2 over a 3-component strided field (b optional, complex64)
__global__ void __launch_bounds__(kKThreads) k_norm2_c128(const double2* __restrict__ a, long acs,
                                                         const float2* __restrict__ b, long bcs, long n,
                                                         double2* __restrict__ part, unsigned* __restrict__ counter,
                                                         double2* __restrict__ out) {
  __shared__ double2 red[kKThreads / 32];
  double2 acc = make_double2(0.0, 0.0);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * n; i += (long)gridDim.x * blockDim.x) {
    const long c = i / n, e = i % n;
    double2 v = a[c * acs + e];
    if (b) v = v + to_c64(b[c * bcs + e]);
    acc.x += v.x * v.x + v.y * v.y;
  }
  const double2 s = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
  if (!arrive_last(counter, gridDim.x)) return;
  const double2 tot = sum_partials(part, gridDim.x, red);
  if (threadIdx.x == 0) {
    *out = tot;
    *counter = 0u;
  }
}

// ------------------------------------------------------------------ launchers
template <typename T>
cudaError_t Krylov<T>::dots(const C<T>* V, long ld, int nv, const C<T>* w, long n, bool with_norm, double2* out,
                            double2* acc, const int* skip, const RedScratch& sc, cudaStream_t s) {
  if (nv < 1 || nv > kMaxBasis) return cudaErrorInvalidValue;
  // blocks the GPU holds at once for this kernel: the groups' blocks together fill one wave
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dots<T>, kKThreads, 0);
    cudaGetLastError();
    return sms * per_sm > 0 ? sms * per_sm : kRedBlocks;
  }();
  const int ng = (nv + kDotGroup - 1) / kDotGroup;
  const int gx = std::max(1, std::min(krylov_blocks(n), resident / ng));
  dim3 grd(gx, ng);
  k_dots<T><<<grd, kKThreads, 0, s>>>(V, ld, nv, w, n, with_norm ? 1 : 0, sc.part, sc.counters, out, acc, skip);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::update(const C<T>* V, long ld, int nv, const double2* h, C<T>* w, long n, double2* out_norm,
                              const double2* ref, double eta2, int* flag, const int* skip, const RedScratch& sc,
                              cudaStream_t s) {
  if (nv < 1 || nv > kMaxBasis) return cudaErrorInvalidValue;
  k_update<T><<<krylov_blocks(n), kKThreads, 0, s>>>(V, ld, nv, h, w, n, sc.part, sc.counters + kCounterUpdate,
                                                      out_norm, ref, eta2, flag, skip);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::combine(const C<T>* V, long ld, int nv, const double2* y, C<T>* x, long n, cudaStream_t s,
                               const int* nv_dev) {
  if (nv > kMaxBasis) return cudaErrorInvalidValue;
  k_combine<T><<<krylov_blocks(n) * 2, kKThreads, 0, s>>>(V, ld, nv, y, x, n, nv_dev);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::scale(const C<T>* src, C<T>* dst, long n, const double2* nrm2, double host_scale,
                             cudaStream_t s) {
  k_scale<T><<<krylov_blocks(n) * 2, kKThreads, 0, s>>>(src, dst, n, nrm2, host_scale);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::norm2(const C<T>* v, long n, double2* out, const RedScratch& sc, cudaStream_t s) {
  k_norm2<T><<<krylov_blocks(n), kKThreads, 0, s>>>(v, n, nullptr, nullptr, sc.part, sc.counters + kCounterNorm, out);
  return cudaGetLastError();
}
template <typename T>
cudaError_t Krylov<T>::rsub(const C<T>* b, C<T>* y, long n, double2* out, const RedScratch& sc, cudaStream_t s) {
  k_norm2<T><<<krylov_blocks(n), kKThreads, 0, s>>>(nullptr, n, b, y, sc.part, sc.counters + kCounterNorm, out);
  return cudaGetLastError();
}
template struct Krylov<float>;
template struct Krylov<double>;

// ---------------------------------------------------------------- GMRES control on the device
// One thread each: the work is O(m) (rotations) or O(m^2) (back substitution) FP64 operations.
namespace {
__device__ __forceinline__ double2 zc(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return zc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return zc(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return zc(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return zc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double zabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return zc(a.x * s, a.y * s); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = zabs2(b);
  return zc((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
}  // namespace

__global__ void k_gm_init(GmState* st, const double2* nrm2, cudaGraphConditionalHandle outer) {
  const double b2 = nrm2->x;
  st->bnorm = b2 > 0.0 ? sqrt(b2) : 0.0;
  st->beta = st->bnorm;
  st->iters = st->cycles = st->reorth = st->j = st->jd = 0;
  st->rel = st->bnorm > 0.0 ? 1.0 : 0.0;
  st->est = st->rel;
  st->status = st->bnorm > 0.0 ? 0 : 1;
  cudaGraphSetConditional(outer, st->bnorm > 0.0 ? 1u : 0u);
}

__global__ void k_gm_cycle(GmState* st, const GmSteps steps) {
  st->j = 0;
  st->g[0] = zc(st->beta, 0.0);
  for (int i = 1; i <= st->m; ++i) st->g[i] = zc(0.0, 0.0);
  for (int k = 0; k < steps.m; ++k) cudaGraphSetConditional(steps.h[k], k == 0 ? 1u : 0u);
}

__global__ void k_gm_step(GmState* st, int j, const double2* __restrict__ h, const double2* __restrict__ nrm2,
                          const int* __restrict__ reorth_flag, cudaGraphConditionalHandle next, int has_next) {
  constexpr int M = kGmMaxM;
  double2* H = st->H;
  for (int i = 0; i <= j; ++i) H[i * M + j] = h[i];
  const double hn = sqrt(fmax(nrm2->x, 0.0));
  H[(j + 1) * M + j] = zc(hn, 0.0);
  if (reorth_flag && *reorth_flag) st->reorth++;
  for (int i = 0; i < j; ++i) {
    const double2 hij = H[i * M + j], hi1 = H[(i + 1) * M + j];
    const double2 t = zadd(zmul(st->cs[i], hij), zmul(st->sn[i], hi1));
    H[(i + 1) * M + j] = zadd(zmul(zc(-st->sn[i].x, st->sn[i].y), hij), zmul(zconj(st->cs[i]), hi1));
    H[i * M + j] = t;
  }
  const double2 a = H[j * M + j], d = H[(j + 1) * M + j];
  const double den = sqrt(zabs2(a) + zabs2(d));
  st->cs[j] = den != 0.0 ? zscale(zconj(a), 1.0 / den) : zc(1.0, 0.0);
  st->sn[j] = den != 0.0 ? zscale(zconj(d), 1.0 / den) : zc(0.0, 0.0);
  H[j * M + j] = zadd(zmul(st->cs[j], a), zmul(st->sn[j], d));
  H[(j + 1) * M + j] = zc(0.0, 0.0);
  const double2 gj = st->g[j];
  st->g[j + 1] = zmul(zc(-st->sn[j].x, st->sn[j].y), gj);
  st->g[j] = zmul(st->cs[j], gj);
  st->iters++;
  st->j = j + 1;
  const double est = sqrt(zabs2(st->g[j + 1])) / st->bnorm;
  st->est = est;
  const bool stop = !(est > st->tol) || hn == 0.0 || st->iters >= st->max_it || j + 1 >= st->m;
  if (!isfinite(est)) st->status = 3;
  if (has_next) cudaGraphSetConditional(next, (stop || st->status == 3) ? 0u : 1u);
}

__global__ void k_gm_solve(GmState* st, double2* __restrict__ y_out) {
  constexpr int M = kGmMaxM;
  const int jd = st->status == 3 ? 0 : st->j;
  for (int i = jd - 1; i >= 0; --i) {
    double2 acc = st->g[i];
    for (int k = i + 1; k < jd; ++k) acc = zsub(acc, zmul(st->H[i * M + k], st->y[k]));
    st->y[i] = zdiv(acc, st->H[i * M + i]);
  }
  for (int i = 0; i < jd; ++i) y_out[i] = st->y[i];
  st->jd = jd;
  if (st->cycles < kGmMaxCycles) st->cyc_len[st->cycles] = st->j;
}

__global__ void k_gm_restart(GmState* st, const double2* __restrict__ nrm2, cudaGraphConditionalHandle outer) {
  const double beta = sqrt(fmax(nrm2->x, 0.0));
  st->beta = beta;
  st->rel = beta / st->bnorm;
  st->cycles++;
  unsigned more = 1u;
  if (!isfinite(st->rel) || st->status == 3) {
    st->status = 3;
    more = 0u;
  } else if (st->rel <= st->tol) {
    st->status = 1;
    more = 0u;
  } else if (st->iters >= st->max_it || beta == 0.0 || st->cycles >= st->max_it) {
    st->status = 2;
    more = 0u;
  }
  cudaGraphSetConditional(outer, more);
}

cudaError_t gm_init(GmState* st, const double2* nrm2, cudaGraphConditionalHandle outer, cudaStream_t s) {
  k_gm_init<<<1, 1, 0, s>>>(st, nrm2, outer);
  return cudaGetLastError();
}
cudaError_t gm_cycle(GmState* st, const GmSteps& steps, cudaStream_t s) {
  if (steps.m < 1 || steps.m > kGmMaxM) return cudaErrorInvalidValue;
  k_gm_cycle<<<1, 1, 0, s>>>(st, steps);
  return cudaGetLastError();
}
cudaError_t gm_step(GmState* st, int j, const double2* h, const double2* nrm2, const int* reorth_flag,
                    cudaGraphConditionalHandle next, bool has_next, cudaStream_t s) {
  k_gm_step<<<1, 1, 0, s>>>(st, j, h, nrm2, reorth_flag, next, has_next ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t gm_solve(GmState* st, double2* y_out, cudaStream_t s) {
  k_gm_solve<<<1, 1, 0, s>>>(st, y_out);
  return cudaGetLastError();
}
cudaError_t gm_restart(GmState* st, const double2* nrm2, cudaGraphConditionalHandle outer, cudaStream_t s) {
  k_gm_restart<<<1, 1, 0, s>>>(st, nrm2, outer);
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
cudaError_t launch_add_diff_c64(float2* acc, const float2* a, const float2* b, long n3, cudaStream_t s) {
  k_add_diff_c64<<<egrid(n3 / 3 + 1), 256, 0, s>>>(acc, a, b, n3);
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
cudaError_t launch_norm2_c128(const double2* a, long acs, const float2* b, long bcs, long n, double2* out,
                              const RedScratch& sc, cudaStream_t s) {
  k_norm2_c128<<<kRedBlocks, kKThreads, 0, s>>>(a, acs, b, bcs, n, sc.part, sc.counters + kCounterNorm, out);
  return cudaGetLastError();
}

}  // namespace ie
