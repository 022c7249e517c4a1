// P3 with warp-resident pencils: z-FFT of the three components, 3x3 Green product, inverse z-FFT.
//
// The same computation as k_p3_spectral (eq. 10 along z, in the mixed (kx, ky, z) domain), organised
// so that no block-wide barrier is needed: all TT = L/16 threads of a pencil sit in one warp (W = 32/TT
// neighbouring lanes kx per warp), each warp exchanges its FFT stages through its own shared-memory
// slot with __syncwarp, and the three forward spectra stay in the registers of the thread that
// computed them (thread t holds kz = t + TT*m, m = 0..15, for all three components), so the Green
// product reads no shared memory. A block is NW warps on NW*W neighbouring lanes, which keeps the
// global rows of a block together in 8*NW*W-byte segments.
//
// Green octant and signs as in k_p3_spectral: with s_a = +-1 the side of axis a,
// Y_p = sum_q s_p s_q F_pq(|k|) J_q, so the off-diagonal octant values are used with the sign
// products s_x s_y, s_x s_z, s_y s_z; s_x and s_y are fixed per thread, s_z per register (m < E/2 is
// the lower half of the z frequencies, the Nyquist row may take either side).
#pragma once
#include "fft.cuh"

namespace ie {

template <int L> struct P3WCfg {
  static constexpr int E = Plan<float, L>::E;   // 16 for L >= 16
  static constexpr int TT = Plan<float, L>::TT;  // threads per pencil
  static constexpr int W = 32 / TT;              // pencils (lanes) per warp
  static constexpr int NW = 4;                   // warps per block
  static constexpr int LANES = NW * W;           // lanes per block
  static constexpr int SLOT = RowSM<float>::words(L);  // complex words per pencil slot
};

template <int L>
__global__ void __launch_bounds__(128, 3) k_p3_warp(const float2* __restrict__ Bin, int in_cs, int nzs, int os,
                                                    float2* __restrict__ Bout, int out_cs, int nzt, int ot,
                                                    const float2* __restrict__ G, int Lx, int Ly,
                                                    const float2* __restrict__ tw) {
  using Cfg = P3WCfg<L>;
  constexpr int E = Cfg::E, TT = Cfg::TT, W = Cfg::W;
  static_assert(TT <= 32 && 32 % TT == 0, "a pencil must fit in one warp");
  __shared__ float2 smem[Cfg::NW * W * Cfg::SLOT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane / TT, t = lane % TT;
  const int kx = blockIdx.x * Cfg::LANES + warp * W + p, ky = blockIdx.y;
  const bool act = kx < Lx;
  const int plane = Ly * Lx, off = ky * Lx + (act ? kx : 0);
  RowSM<float> sm{smem + (warp * W + p) * Cfg::SLOT};
  float2 J[3][E];
  // forward z-FFT of each component (the source rows sit at pencil positions [os, os + nzs))
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int z = t + TT * m - os;
      J[c][m] = (act && z >= 0 && z < nzs) ? __ldg(Bin + c * in_cs + z * plane + off) : make_float2(0.f, 0.f);
    }
    pencil_fft<float, L, -1, RowSM<float>, WarpSync>(J[c], t, sm, tw);
  }
  // Green product in registers
  {
    const int ox = Lx / 2 + 1, oy = Ly / 2 + 1;
    const int ocs = (L / 2 + 1) * oy * ox, ozs = oy * ox;
    const bool xlo = kx <= Lx / 2, ylo = ky <= Ly / 2;
    const int ix = act ? (xlo ? kx : Lx - kx) : 0, iy = ylo ? ky : Ly - ky;
    const float sx = xlo ? 1.f : -1.f, sy = ylo ? 1.f : -1.f, sxy = sx * sy;
    const float2* gb = G + iy * ox + ix;
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const bool zlo = (E == 1) || (m < E / 2);
      const int kz = t + TT * m, iz = zlo ? kz : L - kz;
      const float2* g = gb + iz * ozs;
      const float2 gxx = __ldg(g), gyy = __ldg(g + ocs), gzz = __ldg(g + 2 * ocs);
      const float2 gxy = __ldg(g + 3 * ocs), gxz = __ldg(g + 4 * ocs), gyz = __ldg(g + 5 * ocs);
      const float sxz = zlo ? sx : -sx, syz = zlo ? sy : -sy;
      const float2 j0 = J[0][m], j1 = J[1][m], j2 = J[2][m];
      const float2 a01 = cmul(gxy, j1), a02 = cmul(gxz, j2), a12 = cmul(gyz, j2);
      const float2 a10 = cmul(gxy, j0), a20 = cmul(gxz, j0), a21 = cmul(gyz, j1);
      float2 y0 = cmul(gxx, j0), y1 = cmul(gyy, j1), y2 = cmul(gzz, j2);
      y0.x = fmaf(sxy, a01.x, fmaf(sxz, a02.x, y0.x));
      y0.y = fmaf(sxy, a01.y, fmaf(sxz, a02.y, y0.y));
      y1.x = fmaf(sxy, a10.x, fmaf(syz, a12.x, y1.x));
      y1.y = fmaf(sxy, a10.y, fmaf(syz, a12.y, y1.y));
      y2.x = fmaf(sxz, a20.x, fmaf(syz, a21.x, y2.x));
      y2.y = fmaf(sxz, a20.y, fmaf(syz, a21.y, y2.y));
      J[0][m] = y0;
      J[1][m] = y1;
      J[2][m] = y2;
    }
  }
  // inverse z-FFT and crop to the target rows [ot, ot + nzt)
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pencil_fft<float, L, +1, RowSM<float>, WarpSync>(J[c], t, sm, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int z = t + TT * m - ot;
        if (z >= 0 && z < nzt) Bout[c * out_cs + z * plane + off] = J[c][m];
      }
    }
  }
}

}  // namespace ie
