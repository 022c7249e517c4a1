// 3D Fourier neural operator used as a learned initial guess for the sub-domain solves (an extension
// of the method: the paper's own warm start is the previous sweep's field). Forward, backward, loss and
// Adam, all on the GPU.
//
//   input a (B, N^3, Cin) -> lift P -> L x [ v <- act(v W_l + w_l + K_l v) ] -> GELU(v Q1 + q1) Q2 + q2
//   K_l v = S( R_l * T v ): T is the truncated DFT of the real field (kz in 0..M-1; ky, kx in
//   {0..M-1} U {N-M..N-1}), R_l one complex C x C matrix per retained mode, S the truncated real
//   inverse (weights c_0 = 1, c_kz = 2; factor N^-3). act = GELU (erf form) except after the last layer.
//
// Activations are channels-last, (b, p, c) with p = (z N + y) N + x. The saved activations and the
// spectral weights are stored in S (float, or bf16 for training/inference); every sum accumulates in FP32.
// Parameter vector (FP32, flat): P, p, W_0..W_{L-1}, w_0..w_{L-1}, R_0..R_{L-1} (complex, [kz][ky][kx][i][o]),
// Q1, q1, Q2, q2 — the order and layouts of the CPU reference.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "ie_fno.h"
#include "tcgen05.cuh"

namespace ie {
namespace fnok {

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16(v); }
__device__ __forceinline__ float2 ldc(const float2* p) { return *p; }
__device__ __forceinline__ float2 ldc(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
__device__ __forceinline__ void stc(float2* p, float2 v) { *p = v; }
__device__ __forceinline__ void stc(__nv_bfloat162* p, float2 v) { *p = __float22bfloat162_rn(v); }
template <typename S> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<__nv_bfloat16> { using type = __nv_bfloat162; };

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// ------------------------------------------------------------------ one-axis truncated DFT
// out[b][o][k][i] = scale * sum_n in[b][o][n][i] * w(f) * exp(sgn 2 pi i f s / N), where along the
// transformed axis one side is spatial (s) and the other a retained mode with frequency f.
struct AxisArgs {
  long in_b, in_o, in_n, out_b, out_o, out_k;
  int nb, nouter, ninner, lin, lout, N, M;
  int fwd;        // 1: n spatial, k a mode; 0: n a mode, k spatial
  int xy_modes;   // mode index -> frequency: 0 identity (z), 1 the two-ended list (x, y)
  int zweight;    // multiply by c_f (1 for f = 0, else 2)
  float sgn, scale;
};
__device__ __forceinline__ int mode_freq(int idx, const AxisArgs& a) {
  return a.xy_modes ? (idx < a.M ? idx : a.N - 2 * a.M + idx) : idx;
}

template <typename InT, bool IN_CPLX, typename OutT, bool OUT_CPLX>
__global__ void __launch_bounds__(256) k_axis_dft(const InT* __restrict__ in, OutT* __restrict__ out, AxisArgs a) {
  __shared__ float2 tw[256];
  for (int q = threadIdx.x; q < a.N; q += blockDim.x) {
    float s, c;
    sincospif(2.0f * (float)q / (float)a.N, &s, &c);
    tw[q] = make_float2(c, a.sgn * s);
  }
  __syncthreads();
  const long total = (long)a.nb * a.nouter * a.lout * a.ninner;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % a.ninner);
    long r = idx / a.ninner;
    const int k = (int)(r % a.lout);
    r /= a.lout;
    const int o = (int)(r % a.nouter);
    const int b = (int)(r / a.nouter);
    const InT* src = in + b * a.in_b + o * a.in_o + i;
    float2 acc = make_float2(0.f, 0.f);
    const int fk = a.fwd ? mode_freq(k, a) : k;
    for (int n = 0; n < a.lin; ++n) {
      const int f = a.fwd ? fk : mode_freq(n, a);
      const int sidx = a.fwd ? n : k;
      const float2 w = tw[(f * sidx) % a.N];
      const float cw = (a.zweight && f != 0) ? 2.f : 1.f;
      if constexpr (IN_CPLX) {
        const float2 v = ldc(src + n * a.in_n);
        acc.x += cw * (v.x * w.x - v.y * w.y);
        acc.y += cw * (v.x * w.y + v.y * w.x);
      } else {
        const float v = ldf(src + n * a.in_n);
        acc.x += cw * v * w.x;
        acc.y += cw * v * w.y;
      }
    }
    OutT* dst = out + b * a.out_b + o * a.out_o + (long)k * a.out_k + i;
    if constexpr (OUT_CPLX)
      stc(dst, make_float2(a.scale * acc.x, a.scale * acc.y));
    else
      stf(dst, a.scale * acc.x);
  }
}

// ------------------------------------------------------------------ per-mode channel mixing
// fwd:  Y[b][m][o] = sum_i X[b][m][i] R[m][i][o]
template <typename RS>
__global__ void k_mix_fwd(const float2* __restrict__ X, const RS* __restrict__ R, float2* __restrict__ Y, int B,
                          long nm, int C) {
  const long total = (long)B * nm * C;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % C);
    const long bm = idx / C, m = bm % nm;
    const float2* x = X + bm * C;
    const RS* r = R + m * C * C + o;
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < C; ++i) {
      const float2 xv = x[i], rv = ldc(r + (long)i * C);
      acc.x += xv.x * rv.x - xv.y * rv.y;
      acc.y += xv.x * rv.y + xv.y * rv.x;
    }
    Y[idx] = acc;
  }
}
// input adjoint:  dX[b][m][i] = sum_o conj(R[m][i][o]) dY[b][m][o]
template <typename RS>
__global__ void k_mix_bwd_x(const float2* __restrict__ dY, const RS* __restrict__ R, float2* __restrict__ dX, int B,
                            long nm, int C) {
  const long total = (long)B * nm * C;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % C);
    const long bm = idx / C, m = bm % nm;
    const float2* dy = dY + bm * C;
    const RS* r = R + (m * C + i) * C;
    float2 acc = make_float2(0.f, 0.f);
    for (int o = 0; o < C; ++o) {
      const float2 g = dy[o], rv = ldc(r + o);
      acc.x += rv.x * g.x + rv.y * g.y;
      acc.y += rv.x * g.y - rv.y * g.x;
    }
    dX[idx] = acc;
  }
}
// weight gradient:  gR[m][i][o] += sum_b dY[b][m][o] conj(X[b][m][i])
__global__ void k_mix_grad(const float2* __restrict__ dY, const float2* __restrict__ X, float2* __restrict__ gR, int B,
                           long nm, int C) {
  const long total = nm * C * C;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % C), i = (int)((idx / C) % C);
    const long m = idx / ((long)C * C);
    float2 acc = gR[idx];
    for (int b = 0; b < B; ++b) {
      const float2 g = dY[((long)b * nm + m) * C + o], x = X[((long)b * nm + m) * C + i];
      acc.x += g.x * x.x + g.y * x.y;
      acc.y += g.y * x.x - g.x * x.y;
    }
    gR[idx] = acc;
  }
}

// ------------------------------------------------------------------ pointwise channel maps
// Y[r][o] = sum_i f(X[r][i]) Mt[i][o] + bias[o] (+ add[r][o]); f = GELU when xgelu. Stores the value in
// Ypre (if not null) and act(value) in Yact (act = GELU when ygelu).
template <typename SX, typename SY, typename SA>
__global__ void k_mm_fwd(const SX* __restrict__ X, int I, const float* __restrict__ Mt, const float* __restrict__ bias,
                         const SA* __restrict__ add, SY* __restrict__ Ypre, SY* __restrict__ Yact, float* __restrict__ Yf,
                         int O, long rows, int xgelu, int ygelu) {
  const long total = rows * O;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int o = (int)(idx % O);
    const long r = idx / O;
    const SX* x = X + r * I;
    float acc = bias[o];
    for (int i = 0; i < I; ++i) {
      float xv = ldf(x + i);
      if (xgelu) xv = gelu(xv);
      acc += xv * Mt[i * O + o];
    }
    if (add) acc += ldf(add + idx);
    if (Ypre) stf(Ypre + idx, acc);
    if (Yact) stf(Yact + idx, ygelu ? gelu(acc) : acc);
    if (Yf) Yf[idx] = acc;
  }
}
// 16 consecutive values, 16-byte aligned: BF16 as two 16-byte stores, FP32 as four
__device__ __forceinline__ void st16(__nv_bfloat16* p, const float (&v)[16]) {
  uint4 q[2];
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(q);
#pragma unroll
  for (int j = 0; j < 8; ++j) h[j] = __float22bfloat162_rn(make_float2(v[2 * j], v[2 * j + 1]));
  reinterpret_cast<uint4*>(p)[0] = q[0];
  reinterpret_cast<uint4*>(p)[1] = q[1];
}
__device__ __forceinline__ void st16(float* p, const float (&v)[16]) {
#pragma unroll
  for (int j = 0; j < 4; ++j)
    reinterpret_cast<float4*>(p)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}

// The same map on the tensor cores, for BF16 X with I a multiple of 16 (16 <= I <= 128) and O <= 128:
// tcgen05 MMAs of kind::f16 (BF16 operands, FP32 accumulation in tensor memory), M = 128 rows per tile,
// N = O rounded up to 16, K = 16 per instruction. A persistent block of 128 threads keeps Mt (BF16,
// transposed to O x I, K-major) in shared memory; per tile of 128 rows it loads X (GELU applied when
// xgelu), one thread issues the I/16 MMAs and commits them to an mbarrier, every thread waits for it
// (bounded: a timeout sets *err, waits once more and ends the loop; the block always frees its tensor
// memory), then thread r reads row r of the product from tensor memory and writes the epilogue.
constexpr int kTcRows = 128;

template <typename SY>
__global__ void __launch_bounds__(kTcRows) k_mm_fwd_tc(const __nv_bfloat16* __restrict__ X, int I,
                                                     const float* __restrict__ Mt, const float* __restrict__ bias,
                                                     const float* __restrict__ add, SY* __restrict__ Ypre,
                                                     SY* __restrict__ Yact, float* __restrict__ Yf, int O, int Npad,
                                                     unsigned ncols, long rows, int xgelu, int ygelu,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  unsigned char* As = tc_dyn;                                // kTcRows x I BF16, K-major core matrices
  unsigned char* Bs = tc_dyn + (size_t)kTcRows * I * 2;      // Npad x I BF16
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)Npad * I * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_fence_init();
  }
  __syncwarp();  // the warp-wide (aligned) allocation below runs converged
  if (warp == 0) {
    tmem_alloc(tslot, ncols);
    tmem_relinquish();
  }
  for (int q = tid; q < Npad * I; q += kTcRows) {  // B = Mt^T in BF16, rows o >= O zero
    const int o = q / I, i = q % I;
    const float v = o < O ? Mt[i * O + o] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(Bs + kmajor_offset(o, i, I)) = __float2bfloat16(v);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_bf16_f32(kTcRows, Npad);
  const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs), sbo = (uint32_t)(I >> 3) << 7;
  const long ntiles = (rows + kTcRows - 1) / kTcRows;
  const int cpr = I >> 3;  // 16-byte chunks (8 BF16) per row
  unsigned phase = 0;
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long r0 = tile * kTcRows;
    for (int q = tid; q < kTcRows * cpr; q += kTcRows) {
      const int m = q / cpr, kc = q % cpr;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (r0 + m < rows) {
        v = *reinterpret_cast<const uint4*>(X + (r0 + m) * I + kc * 8);
        if (xgelu) {
          __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 fv = __bfloat1622float2(h[j]);
            fv.x = gelu(fv.x);
            fv.y = gelu(fv.y);
            h[j] = __float22bfloat162_rn(fv);
          }
        }
      }
      *reinterpret_cast<uint4*>(As + kmajor_offset(m, kc * 8, I)) = v;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int s = 0; s < I / 16; ++s)
        tc_mma_bf16(tmem, smem_desc(a0 + s * 256, 128, sbo), smem_desc(b0 + s * 256, 128, sbo), idesc, s > 0);
      tc_commit(bar);
    }
    if (!__syncthreads_and(mbar_wait(bar, phase))) {
      if (tid == 0) atomicExch(err, 1);
      mbar_wait(bar, phase);  // once more, bounded, before the tensor memory is freed
      break;
    }
    phase ^= 1u;
    tc_fence_after();
    const long r = r0 + tid;  // warp w owns tensor-memory lanes (rows) 32w .. 32w + 31
    for (int c0 = 0; c0 < Npad; c0 += 16) {
      float d[16];
      __syncwarp();  // the warp-wide (aligned) load runs converged
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, d);
      if (r < rows && O % 16 == 0) {  // 16 whole columns: vector loads and stores (16-byte aligned)
        const long idx = r * O + c0;
        float acc[16], act16[16];
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const float4 bv = *reinterpret_cast<const float4*>(bias + c0 + j);
          acc[j] = d[j] + bv.x;
          acc[j + 1] = d[j + 1] + bv.y;
          acc[j + 2] = d[j + 2] + bv.z;
          acc[j + 3] = d[j + 3] + bv.w;
          if (add) {
            const float4 av = *reinterpret_cast<const float4*>(add + idx + j);
            acc[j] += av.x;
            acc[j + 1] += av.y;
            acc[j + 2] += av.z;
            acc[j + 3] += av.w;
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) act16[j] = ygelu ? gelu(acc[j]) : acc[j];
        if (Ypre) st16(Ypre + idx, acc);
        if (Yact) st16(Yact + idx, act16);
        if (Yf) st16(Yf + idx, acc);
      } else if (r < rows) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int o = c0 + j;
          if (o < O) {
            const long idx = r * O + o;
            float acc = d[j] + bias[o];
            if (add) acc += add[idx];
            if (Ypre) stf(Ypre + idx, acc);
            if (Yact) stf(Yact + idx, ygelu ? gelu(acc) : acc);
            if (Yf) Yf[idx] = acc;
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // every read of this tile's product precedes the next tile's MMAs
  }
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem, ncols);
  }
}

// dX[r][i] = (sum_o dY[r][o] Mt[i][o] + add[r][i]) * (zgelu ? gelu'(Z[r][i]) : 1)
template <typename SZ>
__global__ void k_mm_bwd_x(const float* __restrict__ dY, int O, const float* __restrict__ Mt,
                           const float* __restrict__ add, const SZ* __restrict__ Z, float* __restrict__ dX, int I,
                           long rows, int zgelu) {
  const long total = rows * I;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % I);
    const long r = idx / I;
    const float* dy = dY + r * O;
    float acc = add ? add[idx] : 0.f;
    for (int o = 0; o < O; ++o) acc += dy[o] * Mt[i * O + o];
    if (zgelu) acc *= gelu_grad(ldf(Z + idx));
    dX[idx] = acc;
  }
}
// G[i][o] += sum_r f(X[r][i]) dY[r][o],  gb[o] += sum_r dY[r][o]; f = GELU when xgelu.
// Each block sums a run of rows for every (i, o) it owns, then adds into G once.
template <typename SX>
__global__ void __launch_bounds__(256) k_outer(const SX* __restrict__ X, int I, const float* __restrict__ dY, int O,
                                               long rows, long rows_per_block, float* __restrict__ G,
                                               float* __restrict__ gb, int xgelu) {
  constexpr int TR = 16;
  __shared__ float xs[TR][128], ys[TR][128];
  const int IO = I * O;
  float acc[16];
  float bacc = 0.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  const long r0 = (long)blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  for (long rt = r0; rt < r1; rt += TR) {
    __syncthreads();
    for (int q = threadIdx.x; q < TR * 128; q += blockDim.x) {
      const int rr = q / 128, c = q % 128;
      const long r = rt + rr;
      float xv = 0.f, yv = 0.f;
      if (r < r1) {
        if (c < I) {
          xv = ldf(X + r * I + c);
          if (xgelu) xv = gelu(xv);
        }
        if (c < O) yv = dY[r * O + c];
      }
      xs[rr][c] = xv;
      ys[rr][c] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e < IO) {
        const int i = e / O, o = e % O;
        float s = 0.f;
#pragma unroll
        for (int rr = 0; rr < TR; ++rr) s += xs[rr][i] * ys[rr][o];
        acc[q] += s;
      }
    }
    if (gb && threadIdx.x < O) {
      for (int rr = 0; rr < TR; ++rr) bacc += ys[rr][threadIdx.x];
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int e = threadIdx.x + q * 256;
    if (e < IO) atomicAdd(G + e, acc[q]);
  }
  if (gb && threadIdx.x < O) atomicAdd(gb + threadIdx.x, bacc);
}

// elementwise: dZ = dY * gelu'(Z)
template <typename SZ>
__global__ void k_gelu_bwd(const float* __restrict__ dY, const SZ* __restrict__ Z, float* __restrict__ dZ, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    dZ[i] = dY[i] * gelu_grad(ldf(Z + i));
}

// relative-L2 loss per sample: sums[2b] = |u - t|^2, sums[2b+1] = |t|^2
__global__ void k_loss_sums(const float* __restrict__ u, const float* __restrict__ t, long per, int B,
                            float* __restrict__ sums) {
  __shared__ float red[2][256];
  const int b = blockIdx.y;
  float d2 = 0.f, t2 = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x) {
    const float tv = t[b * per + i], dv = u[b * per + i] - tv;
    d2 += dv * dv;
    t2 += tv * tv;
  }
  red[0][threadIdx.x] = d2;
  red[1][threadIdx.x] = t2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(sums + 2 * b, red[0][0]);
    atomicAdd(sums + 2 * b + 1, red[1][0]);
  }
}
__global__ void k_loss_grad(const float* __restrict__ u, const float* __restrict__ t, long per, int B,
                            const float* __restrict__ sums, float* __restrict__ du) {
  const long n = per * B;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int b = (int)(i / per);
    const float nd = sqrtf(fmaxf(sums[2 * b], 1e-30f)), nt = sqrtf(fmaxf(sums[2 * b + 1], 1e-30f));
    du[i] = (u[i] - t[i]) / (nd * nt * (float)B);
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi, v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}
template <typename S>
__global__ void k_to_storage(const float* __restrict__ src, S* __restrict__ dst, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    stf(dst + i, src[i]);
}
// Warm-start features on an n^3 grid with N cells (fields complex128 [3][N], conductivity [N][6]).
// |b| in FP64 by one block: bn[0] = sqrt(sum |b|^2)
__global__ void __launch_bounds__(1024) k_bnorm(const double2* __restrict__ b, long n3, double* __restrict__ bn) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (long i = threadIdx.x; i < n3; i += blockDim.x) acc += b[i].x * b[i].x + b[i].y * b[i].y;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) bn[0] = sqrt(red[0]);
}
// a[p] = (sigma6[p][0..5] - sigma0 delta, Re/Im b_c[p] * sqrt(N) / |b|)
__global__ void k_encode(const double* __restrict__ s6, double sigma0, const double2* __restrict__ b, long N,
                         const double* __restrict__ bn, float* __restrict__ a) {
  const double sc = bn[0] > 0.0 ? sqrt((double)N) / bn[0] : 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
    float* ap = a + p * 12;
#pragma unroll
    for (int c = 0; c < 6; ++c) ap[c] = (float)(s6[p * 6 + c] - (c < 3 ? sigma0 : 0.0));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = b[c * N + p];
      ap[6 + 2 * c] = (float)(v.x * sc);
      ap[7 + 2 * c] = (float)(v.y * sc);
    }
  }
}
// t[p] = Re/Im (E_c[p] - b_c[p]) * sqrt(N) / |b|   (the scattered part of the block solution)
__global__ void k_encode_target(const double2* __restrict__ E, const double2* __restrict__ b, long N,
                                const double* __restrict__ bn, float* __restrict__ t) {
  const double sc = bn[0] > 0.0 ? sqrt((double)N) / bn[0] : 0.0;
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 e = E[c * N + p], v = b[c * N + p];
      t[p * 6 + 2 * c] = (float)((e.x - v.x) * sc);
      t[p * 6 + 2 * c + 1] = (float)((e.y - v.y) * sc);
    }
  }
}
// x0_c[p] = b_c[p] + |b| / sqrt(N) * (u[p][2c] + i u[p][2c+1])
__global__ void k_decode(const float* __restrict__ u, const double2* __restrict__ b, long N,
                         const double* __restrict__ bn, double2* __restrict__ x0) {
  const double sc = bn[0] / sqrt((double)N);
  for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < N; p += (long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = b[c * N + p];
      x0[c * N + p] = make_double2(v.x + sc * u[p * 6 + 2 * c], v.y + sc * u[p * 6 + 2 * c + 1]);
    }
  }
}

inline unsigned grid_for(long n) {
  long g = (n + 255) / 256;
  if (g > 152L * 32) g = 152L * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace fnok
}  // namespace ie

using namespace ie;
using namespace ie::fnok;

struct ie_fno {
  int N, M, C, Cin, Cout, H, L, Bmax, storage;
  long Np, nm;  // cells, retained modes per channel
  std::vector<long> off;  // parameter offsets: P p W.. w.. R.. Q1 q1 Q2 q2
  long nparams = 0;
  float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
  void* Rs = nullptr;  // spectral weights in storage precision (L x nm x C x C complex)
  void *v = nullptr, *pre = nullptr, *hp = nullptr;  // saved activations (storage precision)
  float2 *V1 = nullptr, *V2 = nullptr, *V3 = nullptr, *Wm = nullptr;  // spectral intermediates (V3 per layer)
  float *kbuf = nullptr, *dv = nullptr, *dpre = nullptr, *dh = nullptr, *u = nullptr, *du = nullptr, *sums = nullptr;
  int adam_t = 0;
  int tensor_cores = 1;    // BF16 pointwise maps on the tcgen05 path (ie_fno_set_tensor_cores)
  int* tc_err = nullptr;   // mapped pinned flag: a tensor-core kernel's bounded wait gave up
  int nsm = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  ~ie_fno() {
    void* ptrs[] = {params, grads, m1, m2, Rs, v, pre, hp, V1, V2, V3, Wm, kbuf, dv, dpre, dh, u, du, sums};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    if (tc_err) cudaFreeHost(tc_err);
  }
  size_t ssz() const { return storage ? 2 : 4; }
  long rows(int B) const { return (long)B * Np; }
};

namespace {

#define FCK(expr)                                              \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) {                                   \
      f->err = std::string(#expr) + ": " + cudaGetErrorString(_e); \
      return _e == cudaErrorMemoryAllocation ? IE_ENOMEM : IE_ECUDA; \
    }                                                          \
  } while (0)

// The six transforms of one spectral convolution, on (B, N^3, C) activations.
template <typename InT, bool IN_C, typename OutT, bool OUT_C>
cudaError_t axis(ie_fno* f, const InT* in, OutT* out, AxisArgs a) {
  k_axis_dft<InT, IN_C, OutT, OUT_C><<<grid_for((long)a.nb * a.nouter * a.lout * a.ninner), 256, 0, f->stream>>>(in, out, a);
  return cudaGetLastError();
}
AxisArgs base(ie_fno* f, int B) {
  AxisArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nb = B;
  a.N = f->N;
  a.M = f->M;
  a.scale = 1.f;
  return a;
}
// T: real (B, N, N, N, C) -> V3 complex (B, M, 2M, 2M, C); zweight/scale for the adjoint of S
template <typename InT>
cudaError_t forward_T(ie_fno* f, int B, const InT* v, float2* V3, int zweight, float scale) {
  const long N = f->N, M = f->M, C = f->C;
  AxisArgs a = base(f, B);
  a.fwd = 1;
  a.sgn = -1.f;
  // z: in [B][N][N*N*C] real -> V1 [B][M][N*N*C]
  a.in_b = N * N * N * C; a.in_o = 0; a.in_n = N * N * C; a.out_b = M * N * N * C; a.out_o = 0; a.out_k = N * N * C;
  a.nouter = 1; a.ninner = (int)(N * N * C); a.lin = (int)N; a.lout = (int)M; a.xy_modes = 0; a.zweight = zweight;
  a.scale = scale;
  cudaError_t e = axis<InT, false, float2, true>(f, v, f->V1, a);
  if (e != cudaSuccess) return e;
  // y: V1 [B][M][N][N*C] -> V2 [B][M][2M][N*C]
  a.in_b = M * N * N * C; a.in_o = N * N * C; a.in_n = N * C; a.out_b = M * 2 * M * N * C; a.out_o = 2 * M * N * C;
  a.out_k = N * C; a.nouter = (int)M; a.ninner = (int)(N * C); a.lin = (int)N; a.lout = (int)(2 * M); a.xy_modes = 1;
  a.zweight = 0; a.scale = 1.f;
  e = axis<float2, true, float2, true>(f, f->V1, f->V2, a);
  if (e != cudaSuccess) return e;
  // x: V2 [B][M*2M][N][C] -> V3 [B][M*2M][2M][C]
  a.in_b = M * 2 * M * N * C; a.in_o = N * C; a.in_n = C; a.out_b = M * 2 * M * 2 * M * C; a.out_o = 2 * M * C;
  a.out_k = C; a.nouter = (int)(M * 2 * M); a.ninner = (int)C; a.lin = (int)N; a.lout = (int)(2 * M);
  return axis<float2, true, float2, true>(f, f->V2, V3, a);
}
// inverse: W (B, M, 2M, 2M, C) complex -> real (B, N^3, C); zweight/scale select S (1, N^-3) or the
// adjoint of T (0, 1)
cudaError_t inverse_T(ie_fno* f, int B, const float2* W, float* out, int zweight, float scale) {
  const long N = f->N, M = f->M, C = f->C;
  AxisArgs a = base(f, B);
  a.fwd = 0;
  a.sgn = 1.f;
  // x: W [B][M*2M][2M][C] -> V2 [B][M*2M][N][C]
  a.in_b = M * 2 * M * 2 * M * C; a.in_o = 2 * M * C; a.in_n = C; a.out_b = M * 2 * M * N * C; a.out_o = N * C;
  a.out_k = C; a.nouter = (int)(M * 2 * M); a.ninner = (int)C; a.lin = (int)(2 * M); a.lout = (int)N; a.xy_modes = 1;
  cudaError_t e = axis<float2, true, float2, true>(f, W, f->V2, a);
  if (e != cudaSuccess) return e;
  // y: V2 [B][M][2M][N*C] -> V1 [B][M][N][N*C]
  a.in_b = M * 2 * M * N * C; a.in_o = 2 * M * N * C; a.in_n = N * C; a.out_b = M * N * N * C; a.out_o = N * N * C;
  a.out_k = N * C; a.nouter = (int)M; a.ninner = (int)(N * C); a.lin = (int)(2 * M); a.lout = (int)N;
  e = axis<float2, true, float2, true>(f, f->V2, f->V1, a);
  if (e != cudaSuccess) return e;
  // z: V1 [B][M][N*N*C] -> out [B][N][N*N*C] real part
  a.in_b = M * N * N * C; a.in_o = 0; a.in_n = N * N * C; a.out_b = N * N * N * C; a.out_o = 0; a.out_k = N * N * C;
  a.nouter = 1; a.ninner = (int)(N * N * C); a.lin = (int)M; a.lout = (int)N; a.xy_modes = 0; a.zweight = zweight;
  a.scale = scale;
  return axis<float2, true, float, false>(f, f->V1, out, a);
}

template <typename S> S* act(ie_fno* f, void* base_ptr, int l, int B, int ch) {
  return reinterpret_cast<S*>(base_ptr) + (long)l * f->rows(f->Bmax) * ch;
}

// Y = f(X) Mt + bias (+ add) on the tensor cores when the network stores BF16 activations and the shape
// allows it (I a multiple of 16 up to 128, O up to 128); otherwise, or with tensor cores switched off,
// on the CUDA cores (k_mm_fwd).
template <typename SX, typename SY>
cudaError_t mm_fwd(ie_fno* f, const SX* X, int I, const float* Mt, const float* bias, const float* add, SY* Ypre,
                   SY* Yact, float* Yf, int O, long rows, int xgelu, int ygelu) {
  if constexpr (std::is_same<SX, __nv_bfloat16>::value) {
    if (f->tensor_cores && I % 16 == 0 && I >= 16 && I <= 128 && O <= 128 && rows > 0) {
      const int Npad = (O + 15) / 16 * 16;
      unsigned ncols = 32;
      while ((int)ncols < Npad) ncols <<= 1;
      const size_t smem = (size_t)kTcRows * I * 2 + (size_t)Npad * I * 2 + 16;
      static cudaError_t ae = cudaFuncSetAttribute(k_mm_fwd_tc<SY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   96 * 1024);
      if (ae != cudaSuccess) return ae;
      const long ntiles = (rows + kTcRows - 1) / kTcRows;
      const int grid = (int)std::min<long>(ntiles, 3L * std::max(f->nsm, 1));
      int* err = nullptr;
      cudaError_t e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&err), f->tc_err, 0);
      if (e != cudaSuccess) return e;
      k_mm_fwd_tc<SY><<<grid, kTcRows, smem, f->stream>>>(X, I, Mt, bias, add, Ypre, Yact, Yf, O, Npad, ncols, rows,
                                                          xgelu, ygelu, err);
      return cudaGetLastError();
    }
  }
  k_mm_fwd<SX, SY, float><<<grid_for(rows * O), 256, 0, f->stream>>>(X, I, Mt, bias, add, Ypre, Yact, Yf, O, rows,
                                                                     xgelu, ygelu);
  return cudaGetLastError();
}

template <typename S> ie_status fwd_impl(ie_fno* f, int B, const float* a, float* u) {
  using CS = typename Cx<S>::type;
  if (f->tc_err && *reinterpret_cast<volatile int*>(f->tc_err)) {
    *f->tc_err = 0;
    f->err = "a tensor-core kernel's wait for its MMAs reached its limit";
    return IE_ECUDA;
  }
  const long rows = f->rows(B);
  const int C = f->C;
  const float* P = f->params + f->off[0];
  // lift: v_0 = a P + p
  k_mm_fwd<float, S, float><<<grid_for(rows * C), 256, 0, f->stream>>>(a, f->Cin, P, f->params + f->off[1], nullptr,
                                                                       nullptr, act<S>(f, f->v, 0, B, C), nullptr, C,
                                                                       rows, 0, 0);
  FCK(cudaGetLastError());
  for (int l = 0; l < f->L; ++l) {
    S* vl = act<S>(f, f->v, l, B, C);
    float2* V3 = f->V3 + (long)l * B * f->nm * C;
    FCK(forward_T<S>(f, B, vl, V3, 0, 1.f));
    k_mix_fwd<CS><<<grid_for((long)B * f->nm * C), 256, 0, f->stream>>>(
        V3, reinterpret_cast<const CS*>(f->Rs) + (long)l * f->nm * C * C, f->Wm, B, f->nm, C);
    FCK(cudaGetLastError());
    FCK(inverse_T(f, B, f->Wm, f->kbuf, 1, 1.f / ((float)f->N * f->N * f->N)));
    const bool last = (l == f->L - 1);
    FCK((mm_fwd<S, S>(f, vl, C, f->params + f->off[2 + l], f->params + f->off[2 + f->L + l], f->kbuf,
                     act<S>(f, f->pre, l, B, C), act<S>(f, f->v, l + 1, B, C), nullptr, C, rows, 0, last ? 0 : 1)));
  }
  const long oQ1 = f->off[2 + 3 * f->L];
  // head: hp = v_L Q1 + q1 ; u = GELU(hp) Q2 + q2
  FCK((mm_fwd<S, S>(f, act<S>(f, f->v, f->L, B, C), C, f->params + oQ1, f->params + oQ1 + (long)C * f->H, nullptr,
                   reinterpret_cast<S*>(f->hp), nullptr, nullptr, f->H, rows, 0, 0)));
  const long oQ2 = oQ1 + (long)C * f->H + f->H;
  FCK((mm_fwd<S, float>(f, reinterpret_cast<S*>(f->hp), f->H, f->params + oQ2, f->params + oQ2 + (long)f->H * f->Cout,
                       nullptr, nullptr, nullptr, u, f->Cout, rows, 1, 0)));
  return IE_OK;
}

template <typename S> ie_status bwd_impl(ie_fno* f, int B, const float* a, const float* du) {
  using CS = typename Cx<S>::type;
  const long rows = f->rows(B);
  const int C = f->C, H = f->H;
  float* g = f->grads;
  FCK(cudaMemsetAsync(g, 0, sizeof(float) * f->nparams, f->stream));
  const long oQ1 = f->off[2 + 3 * f->L], oQ2 = oQ1 + (long)C * H + H;
  const unsigned ob = (unsigned)((rows + 4095) / 4096);
  S* hp = reinterpret_cast<S*>(f->hp);
  // head: gQ2, gq2 from GELU(hp) and du; dhp = (du Q2^T) * gelu'(hp)
  k_outer<S><<<ob, 256, 0, f->stream>>>(hp, H, du, f->Cout, rows, 4096, g + oQ2, g + oQ2 + (long)H * f->Cout, 1);
  FCK(cudaGetLastError());
  k_mm_bwd_x<S><<<grid_for(rows * H), 256, 0, f->stream>>>(du, f->Cout, f->params + oQ2, nullptr, hp, f->dh, H, rows, 1);
  FCK(cudaGetLastError());
  S* vL = act<S>(f, f->v, f->L, B, C);
  k_outer<S><<<ob, 256, 0, f->stream>>>(vL, C, f->dh, H, rows, 4096, g + oQ1, g + oQ1 + (long)C * H, 0);
  FCK(cudaGetLastError());
  k_mm_bwd_x<float><<<grid_for(rows * C), 256, 0, f->stream>>>(f->dh, H, f->params + oQ1, nullptr, nullptr, f->dv, C,
                                                               rows, 0);
  FCK(cudaGetLastError());
  for (int l = f->L - 1; l >= 0; --l) {
    S* vl = act<S>(f, f->v, l, B, C);
    // dpre = dv * gelu'(pre) except for the last layer
    if (l < f->L - 1) {
      k_gelu_bwd<S><<<grid_for(rows * C), 256, 0, f->stream>>>(f->dv, act<S>(f, f->pre, l, B, C), f->dpre, rows * C);
      FCK(cudaGetLastError());
    } else {
      FCK(cudaMemcpyAsync(f->dpre, f->dv, sizeof(float) * rows * C, cudaMemcpyDeviceToDevice, f->stream));
    }
    k_outer<S><<<ob, 256, 0, f->stream>>>(vl, C, f->dpre, C, rows, 4096, g + f->off[2 + l], g + f->off[2 + f->L + l], 0);
    FCK(cudaGetLastError());
    // adjoint of S: dWm = c_kz N^-3 T(dpre); gR += dWm conj(V3); dV = R^H dWm; kbuf = Re(T^H dV)
    FCK(forward_T<float>(f, B, f->dpre, f->Wm, 1, 1.f / ((float)f->N * f->N * f->N)));
    const float2* V3 = f->V3 + (long)l * B * f->nm * C;
    k_mix_grad<<<grid_for(f->nm * C * C), 256, 0, f->stream>>>(f->Wm, V3, reinterpret_cast<float2*>(g + f->off[2 + 2 * f->L + l]),
                                                                B, f->nm, C);
    FCK(cudaGetLastError());
    k_mix_bwd_x<CS><<<grid_for((long)B * f->nm * C), 256, 0, f->stream>>>(
        f->Wm, reinterpret_cast<const CS*>(f->Rs) + (long)l * f->nm * C * C, f->V3 + (long)f->L * B * f->nm * C, B,
        f->nm, C);
    FCK(cudaGetLastError());
    FCK(inverse_T(f, B, f->V3 + (long)f->L * B * f->nm * C, f->kbuf, 0, 1.f));
    // dv_prev = dpre W^T + kbuf
    k_mm_bwd_x<float><<<grid_for(rows * C), 256, 0, f->stream>>>(f->dpre, C, f->params + f->off[2 + l], f->kbuf,
                                                                 nullptr, f->dv, C, rows, 0);
    FCK(cudaGetLastError());
  }
  // lift: gP += a^T dv_0, gp += sum dv_0
  k_outer<float><<<ob, 256, 0, f->stream>>>(a, f->Cin, f->dv, C, rows, 4096, g + f->off[0], g + f->off[1], 0);
  FCK(cudaGetLastError());
  return IE_OK;
}

ie_status sync_params(ie_fno* f) {
  const long nR = (long)f->L * f->nm * f->C * f->C * 2;
  const float* R = f->params + f->off[2 + 2 * f->L];
  if (f->storage)
    k_to_storage<__nv_bfloat16><<<grid_for(nR), 256, 0, f->stream>>>(R, reinterpret_cast<__nv_bfloat16*>(f->Rs), nR);
  else
    k_to_storage<float><<<grid_for(nR), 256, 0, f->stream>>>(R, reinterpret_cast<float*>(f->Rs), nR);
  FCK(cudaGetLastError());
  return IE_OK;
}

}  // namespace

extern "C" {

ie_status ie_fno_create(int32_t n, int32_t modes, int32_t width, int32_t layers, int32_t cin, int32_t cout,
                        int32_t hidden, int32_t batch_max, int32_t storage, ie_fno** out) {
  if (!out) return IE_EINVAL;
  *out = nullptr;
  if (n < 2 || n > 256 || modes < 1 || 2 * modes > n || width < 1 || width > 128 || layers < 1 || cin < 1 ||
      cin > 128 || cout < 1 || cout > 128 || hidden < 1 || hidden > 128 || batch_max < 1 || (storage != 0 && storage != 1))
    return IE_EINVAL;
  // every weight matrix must fit the 4096 accumulators of one k_outer block
  if ((long)cin * width > 4096 || (long)width * width > 4096 || (long)width * hidden > 4096 || (long)hidden * cout > 4096)
    return IE_EINVAL;
  auto* f = new (std::nothrow) ie_fno();
  if (!f) return IE_ENOMEM;
  f->N = n; f->M = modes; f->C = width; f->L = layers; f->Cin = cin; f->Cout = cout; f->H = hidden;
  f->Bmax = batch_max; f->storage = storage;
  f->Np = (long)n * n * n;
  f->nm = (long)modes * 2 * modes * 2 * modes;
  long o = 0;
  auto push = [&](long sz) { f->off.push_back(o); o += sz; };
  push((long)cin * width); push(width);
  for (int l = 0; l < layers; ++l) push((long)width * width);
  for (int l = 0; l < layers; ++l) push(width);
  for (int l = 0; l < layers; ++l) push(f->nm * width * width * 2);
  push((long)width * hidden); push(hidden); push((long)hidden * cout); push(cout);
  f->nparams = o;
  const long rows = f->rows(batch_max), C = width;
  const size_t s = f->ssz();
  const long nR = (long)layers * f->nm * C * C * 2;
  bool ok = cudaMalloc(&f->params, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&f->grads, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&f->m1, sizeof(float) * o) == cudaSuccess && cudaMalloc(&f->m2, sizeof(float) * o) == cudaSuccess &&
            cudaMalloc(&f->Rs, s * nR) == cudaSuccess &&
            cudaMalloc(&f->v, s * rows * C * (layers + 1)) == cudaSuccess &&
            cudaMalloc(&f->pre, s * rows * C * layers) == cudaSuccess && cudaMalloc(&f->hp, s * rows * hidden) == cudaSuccess &&
            cudaMalloc(&f->V1, sizeof(float2) * batch_max * modes * n * n * C) == cudaSuccess &&
            cudaMalloc(&f->V2, sizeof(float2) * batch_max * modes * 2 * modes * n * C) == cudaSuccess &&
            cudaMalloc(&f->V3, sizeof(float2) * (layers + 1) * batch_max * f->nm * C) == cudaSuccess &&
            cudaMalloc(&f->Wm, sizeof(float2) * batch_max * f->nm * C) == cudaSuccess &&
            cudaMalloc(&f->kbuf, sizeof(float) * rows * C) == cudaSuccess &&
            cudaMalloc(&f->dv, sizeof(float) * rows * C) == cudaSuccess &&
            cudaMalloc(&f->dpre, sizeof(float) * rows * C) == cudaSuccess &&
            cudaMalloc(&f->dh, sizeof(float) * rows * hidden) == cudaSuccess &&
            cudaMalloc(&f->u, sizeof(float) * rows * cout) == cudaSuccess &&
            cudaMalloc(&f->du, sizeof(float) * rows * cout) == cudaSuccess &&
            cudaMalloc(&f->sums, sizeof(float) * 2 * batch_max) == cudaSuccess &&
            cudaMemset(f->m1, 0, sizeof(float) * o) == cudaSuccess && cudaMemset(f->m2, 0, sizeof(float) * o) == cudaSuccess &&
            cudaMemset(f->params, 0, sizeof(float) * o) == cudaSuccess;
  if (!ok) {
    delete f;
    return IE_ENOMEM;
  }
  if (cudaHostAlloc(reinterpret_cast<void**>(&f->tc_err), sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
    f->tc_err = nullptr;
    delete f;
    return IE_ENOMEM;
  }
  *f->tc_err = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&f->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete f;
    return IE_ECUDA;
  }
  *out = f;
  return IE_OK;
}

ie_status ie_fno_set_tensor_cores(ie_fno* f, int32_t on) {
  if (!f || (on != 0 && on != 1)) return IE_EINVAL;
  f->tensor_cores = on;
  return IE_OK;
}

int64_t ie_fno_param_count(const ie_fno* f) { return f ? f->nparams : -1; }

ie_status ie_fno_set_stream(ie_fno* f, void* stream) {
  if (!f) return IE_EINVAL;
  f->stream = reinterpret_cast<cudaStream_t>(stream);
  return IE_OK;
}

ie_status ie_fno_set_params(ie_fno* f, const float* host) {
  if (!f || !host) return IE_EINVAL;
  FCK(cudaMemcpyAsync(f->params, host, sizeof(float) * f->nparams, cudaMemcpyHostToDevice, f->stream));
  FCK(cudaMemsetAsync(f->m1, 0, sizeof(float) * f->nparams, f->stream));
  FCK(cudaMemsetAsync(f->m2, 0, sizeof(float) * f->nparams, f->stream));
  f->adam_t = 0;
  ie_status st = sync_params(f);
  if (st != IE_OK) return st;
  FCK(cudaStreamSynchronize(f->stream));
  return IE_OK;
}

ie_status ie_fno_get_params(ie_fno* f, float* host) {
  if (!f || !host) return IE_EINVAL;
  FCK(cudaMemcpyAsync(host, f->params, sizeof(float) * f->nparams, cudaMemcpyDeviceToHost, f->stream));
  FCK(cudaStreamSynchronize(f->stream));
  return IE_OK;
}

ie_status ie_fno_forward(ie_fno* f, int32_t batch, const float* a_dev, float* u_dev) {
  if (!f || !a_dev || !u_dev || batch < 1 || batch > f->Bmax) return IE_EINVAL;
  return f->storage ? fwd_impl<__nv_bfloat16>(f, batch, a_dev, u_dev) : fwd_impl<float>(f, batch, a_dev, u_dev);
}

ie_status ie_fno_backward(ie_fno* f, int32_t batch, const float* a_dev, const float* du_dev, float* grads_host) {
  if (!f || !a_dev || !du_dev || batch < 1 || batch > f->Bmax) return IE_EINVAL;
  ie_status st = f->storage ? bwd_impl<__nv_bfloat16>(f, batch, a_dev, du_dev) : bwd_impl<float>(f, batch, a_dev, du_dev);
  if (st != IE_OK) return st;
  if (grads_host) {
    FCK(cudaMemcpyAsync(grads_host, f->grads, sizeof(float) * f->nparams, cudaMemcpyDeviceToHost, f->stream));
    FCK(cudaStreamSynchronize(f->stream));
  }
  return IE_OK;
}

ie_status ie_fno_train_step(ie_fno* f, int32_t batch, const float* a_dev, const float* t_dev, float lr, float* loss) {
  if (!f || !a_dev || !t_dev || batch < 1 || batch > f->Bmax || !(lr > 0)) return IE_EINVAL;
  ie_status st = ie_fno_forward(f, batch, a_dev, f->u);
  if (st != IE_OK) return st;
  const long per = f->Np * f->Cout;
  FCK(cudaMemsetAsync(f->sums, 0, sizeof(float) * 2 * batch, f->stream));
  k_loss_sums<<<dim3(64, batch), 256, 0, f->stream>>>(f->u, t_dev, per, batch, f->sums);
  FCK(cudaGetLastError());
  k_loss_grad<<<grid_for(per * batch), 256, 0, f->stream>>>(f->u, t_dev, per, batch, f->sums, f->du);
  FCK(cudaGetLastError());
  st = ie_fno_backward(f, batch, a_dev, f->du, nullptr);
  if (st != IE_OK) return st;
  f->adam_t++;
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<grid_for(f->nparams), 256, 0, f->stream>>>(f->params, f->grads, f->m1, f->m2, f->nparams, lr, b1, b2, 1e-8f,
                                                      1.f - powf(b1, (float)f->adam_t), 1.f - powf(b2, (float)f->adam_t));
  FCK(cudaGetLastError());
  st = sync_params(f);
  if (st != IE_OK) return st;
  if (loss) {
    std::vector<float> h(2 * batch);
    FCK(cudaMemcpyAsync(h.data(), f->sums, sizeof(float) * 2 * batch, cudaMemcpyDeviceToHost, f->stream));
    FCK(cudaStreamSynchronize(f->stream));
    double acc = 0;
    for (int b = 0; b < batch; ++b) acc += std::sqrt(h[2 * b] / std::max(h[2 * b + 1], 1e-30f));
    *loss = (float)(acc / batch);
  }
  return IE_OK;
}

ie_status ie_fno_encode(ie_fno* f, const double* sigma6_dev, double sigma0, const double* b_dev, float* a_dev,
                        double* bnorm_dev) {
  if (!f || !sigma6_dev || !b_dev || !a_dev || !bnorm_dev || f->Cin != 12 || !(sigma0 > 0)) return IE_EINVAL;
  const double2* b = reinterpret_cast<const double2*>(b_dev);
  k_bnorm<<<1, 1024, 0, f->stream>>>(b, 3 * f->Np, bnorm_dev);
  FCK(cudaGetLastError());
  k_encode<<<grid_for(f->Np), 256, 0, f->stream>>>(sigma6_dev, sigma0, b, f->Np, bnorm_dev, a_dev);
  FCK(cudaGetLastError());
  return IE_OK;
}

ie_status ie_fno_encode_target(ie_fno* f, const double* E_dev, const double* b_dev, const double* bnorm_dev,
                               float* t_dev) {
  if (!f || !E_dev || !b_dev || !bnorm_dev || !t_dev || f->Cout != 6) return IE_EINVAL;
  k_encode_target<<<grid_for(f->Np), 256, 0, f->stream>>>(reinterpret_cast<const double2*>(E_dev),
                                                          reinterpret_cast<const double2*>(b_dev), f->Np, bnorm_dev,
                                                          t_dev);
  FCK(cudaGetLastError());
  return IE_OK;
}

ie_status ie_fno_decode(ie_fno* f, const float* u_dev, const double* b_dev, const double* bnorm_dev, double* x0_dev) {
  if (!f || !u_dev || !b_dev || !bnorm_dev || !x0_dev || f->Cout != 6) return IE_EINVAL;
  k_decode<<<grid_for(f->Np), 256, 0, f->stream>>>(u_dev, reinterpret_cast<const double2*>(b_dev), f->Np, bnorm_dev,
                                                   reinterpret_cast<double2*>(x0_dev));
  FCK(cudaGetLastError());
  return IE_OK;
}

const char* ie_fno_last_error(const ie_fno* f) { return f ? f->err.c_str() : "null network"; }

void ie_fno_destroy(ie_fno* f) {
  if (!f) return;
  if (f->stream) cudaStreamSynchronize(f->stream);
  delete f;
}

}  // extern "C"
