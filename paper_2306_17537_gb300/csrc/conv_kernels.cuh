// Pass kernels of the zero-padded FFT convolution G (dsigma x) (eq. 10 of the paper).
//
// Layouts (complex = float2 or double2, x fastest):
//   source field x, output y     [3][nz][ny][nx]      (component stride given per call)
//   contrast dsigma              [6][Nz][ny][nx] real (xx, yy, zz, xy, xz, yz)
//   A (after x-FFT)              [3][nz][ny][Lx]
//   B (after y-FFT)              [3][nz][Ly][Lx]
//   Green spectra (one octant)   [6][Lz/2+1][Ly/2+1][Lx/2+1], already scaled by 1/(Lx Ly Lz)
// Pass order: P1 contrast + x-FFT, P2 y-FFT, P3 z-FFT + 3x3 spectral product + inverse z-FFT,
// P4 inverse y-FFT, P5 inverse x-FFT + crop + epilogue. The zero padding is never stored: a pass
// only loads the valid part of each pencil and only stores the part the next pass needs.
#pragma once
#include "conv.cuh"
#include "fft.cuh"
#include "tma.cuh"

#include <type_traits>

namespace ie {

constexpr int kThreads = 256;

template <typename T, int L> struct RowCfg {  // pencils contiguous in memory (x axis)
  static constexpr int TT = Plan<T, L>::TT;
  static constexpr int P0 = kThreads / TT;
  static constexpr int P = P0 < 1 ? 1 : (P0 > 64 ? 64 : P0);  // pencils per block
};
// Pencils strided, W neighbouring pencils (lanes) per block, W = NT / TT for about NT threads: the
// default tile of 256 threads, a narrower one of 128 and a wider one of 512 (longer contiguous row
// segments) are the autotuner's choices.
template <typename T, int L, int NT = kThreads> struct LaneCfg {
  static constexpr int TT = Plan<T, L>::TT;
  static constexpr int W0 = NT / TT;
  static constexpr int W = W0 < 1 ? 1 : (W0 > 32 ? 32 : W0);
  static constexpr int NTH = W * TT;
  static constexpr size_t kSmem = (size_t)L * W * sizeof(C<T>);
};

// ---------------------------------------------------------------- P1: J = dsigma x, x-FFT
// CONTRACT: the contraction form, where ds holds dsigma M and mt holds M (both [6][...]); the kernel
// then also stores w = M x (the field the epilogue of P5 subtracts the convolution from).
// Each cell's x, tensor (and M) are read once: J_x stays in registers for the first transform, while J_y
// and J_z are parked in their own rows of A (the positions the transform later overwrites; the same
// thread reads them back, and the lines are still in cache) and transformed one after the other, so a
// thread holds one pencil of E values at a time.
template <typename T, int L, bool CONTRACT>
__global__ void __launch_bounds__(kThreads, 3) k_p1_contrast_fftx(
    const FieldC<T>* __restrict__ x, long x_cs, const FieldR<T>* __restrict__ ds, long d_cs,
    C<T>* __restrict__ A, long A_cs, int nx, long nrows, const C<T>* __restrict__ tw,
    const FieldR<T>* __restrict__ mt, FieldC<T>* __restrict__ w, long w_cs) {
  using R = FieldR<T>;
  constexpr int E = Plan<T, L>::E, TT = Plan<T, L>::TT, P = RowCfg<T, L>::P;
  __shared__ C<T> smem[P * RowSM<T>::words(L)];
  const int t = threadIdx.x, p = threadIdx.y;
  const long row = (long)blockIdx.x * P + p;
  const bool act = row < nrows;
  RowSM<T> sm{smem + p * RowSM<T>::words(L)};
  C<T> J[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int i = t + TT * m;
    J[m] = czero<C<T>>();
    if (act && i < nx) {
      const long o = row * nx + i;
      const FieldC<T> x0 = x[o], x1 = x[x_cs + o], x2 = x[2 * x_cs + o];
      if constexpr (CONTRACT) {  // w = M x
        const R mxx = mt[o], myy = mt[d_cs + o], mzz = mt[2 * d_cs + o];
        const R mxy = mt[3 * d_cs + o], mxz = mt[4 * d_cs + o], myz = mt[5 * d_cs + o];
        w[o] = mk<R>(mxx * x0.x + mxy * x1.x + mxz * x2.x, mxx * x0.y + mxy * x1.y + mxz * x2.y);
        w[w_cs + o] = mk<R>(mxy * x0.x + myy * x1.x + myz * x2.x, mxy * x0.y + myy * x1.y + myz * x2.y);
        w[2 * w_cs + o] = mk<R>(mxz * x0.x + myz * x1.x + mzz * x2.x, mxz * x0.y + myz * x1.y + mzz * x2.y);
      }
      // (xx, yy, zz, xy, xz, yz) storage of the symmetric tensor
      const R sxx = ds[o], syy = ds[d_cs + o], szz = ds[2 * d_cs + o];
      const R sxy = ds[3 * d_cs + o], sxz = ds[4 * d_cs + o], syz = ds[5 * d_cs + o];
      J[m] = to_c(mk<R>(sxx * x0.x + sxy * x1.x + sxz * x2.x, sxx * x0.y + sxy * x1.y + sxz * x2.y), T());
      A[A_cs + row * L + i] =
          to_c(mk<R>(sxy * x0.x + syy * x1.x + syz * x2.x, sxy * x0.y + syy * x1.y + syz * x2.y), T());
      A[2 * A_cs + row * L + i] =
          to_c(mk<R>(sxz * x0.x + syz * x1.x + szz * x2.x, sxz * x0.y + syz * x1.y + szz * x2.y), T());
    }
  }
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    if (c > 0) {
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int i = t + TT * m;
        J[m] = (act && i < nx) ? A[c * A_cs + row * L + i] : czero<C<T>>();
      }
    }
    pencil_fft<T, L, -1>(J, t, sm, tw);
    if (act) {
#pragma unroll
      for (int m = 0; m < E; ++m) A[c * A_cs + row * L + t + TT * m] = J[m];
    }
  }
}

// ---------------------------------------------------------------- P5: inverse x-FFT, crop, epilogue
template <typename T, int L, int MODE>
__global__ void __launch_bounds__(kThreads) k_p5_ifftx_epilogue(
    const C<T>* __restrict__ A, long A_cs, int nx, long nrows,
    const FieldC<T>* __restrict__ xin, long x_cs, FieldC<T>* __restrict__ y, long y_cs,
    double2* __restrict__ r, long r_cs, const double2* __restrict__ b, long b_cs,
    const C<T>* __restrict__ tw) {
  constexpr int E = Plan<T, L>::E, TT = Plan<T, L>::TT, P = RowCfg<T, L>::P;
  __shared__ C<T> smem[P * RowSM<T>::words(L)];
  const int t = threadIdx.x, p = threadIdx.y, c = blockIdx.y;
  const long row = (long)blockIdx.x * P + p;
  const bool act = row < nrows;
  RowSM<T> sm{smem + p * RowSM<T>::words(L)};
  C<T> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = act ? A[c * A_cs + row * L + t + TT * m] : czero<C<T>>();
  pencil_fft<T, L, +1>(v, t, sm, tw);
  if (!act) return;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int i = t + TT * m;
    if (i < nx) {
      const long o = row * nx + i;
      if constexpr (MODE == EPI_APPLY) {
        y[c * y_cs + o] = xin[c * x_cs + o] - to_field(v[m]);
      } else if constexpr (MODE == EPI_CONV) {
        y[c * y_cs + o] = to_field(v[m]);
      } else if constexpr (MODE == EPI_ACCUM128) {
        r[c * r_cs + o] = r[c * r_cs + o] + to_c64(v[m]);
      } else {  // EPI_RESID128: r = b - x + G(dsigma x)
        r[c * r_cs + o] = b[c * b_cs + o] - to_c64(xin[c * x_cs + o]) + to_c64(v[m]);
      }
    }
  }
}

// ---------------------------------------------------------------- strided FFT (P2, P4, setup)
// Pencil element e of lane `lane`, batch z, component c sits at c*cs + z*zs + e*es + lane.
template <typename T, int L, int SIGN, int NT>
__global__ void __launch_bounds__(LaneCfg<T, L, NT>::NTH) k_lanes_fft(
    const C<T>* __restrict__ in, long in_cs, long in_zs, long in_es, int n_in,
    C<T>* __restrict__ out, long out_cs, long out_zs, long out_es, int n_out, int nlanes,
    const C<T>* __restrict__ tw) {
  constexpr int E = Plan<T, L>::E, TT = Plan<T, L>::TT, W = LaneCfg<T, L, NT>::W;
  extern __shared__ __align__(16) unsigned char lanes_dyn[];
  C<T>* smem = reinterpret_cast<C<T>*>(lanes_dyn);
  const int w = threadIdx.x, t = threadIdx.y;
  const long z = blockIdx.y, c = blockIdx.z;
  const int lane = blockIdx.x * W + w;
  const bool act = lane < nlanes;
  LaneSM<T, W> sm{smem + w};
  const C<T>* src = in + c * in_cs + z * in_zs + lane;
  C<T> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int e = t + TT * m;
    v[m] = (act && e < n_in) ? src[(long)e * in_es] : czero<C<T>>();
  }
  pencil_fft<T, L, SIGN>(v, t, sm, tw);
  if (!act) return;
  C<T>* dst = out + c * out_cs + z * out_zs + lane;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int e = t + TT * m;
    if (e < n_out) dst[(long)e * out_es] = v[m];
  }
}

// ---------------------------------------------------------------- P3: z-FFT, Green product, inverse
// B holds planes of Ly*Lx; the source occupies pencil positions [os, os + nzs), the target is read
// back from [ot, ot + nzt). With os = ot = 0 this is a block's own convolution; with the whole-domain
// spectra and os/ot the blocks' z offsets it is the interaction between two sub-domains.
// The three forward spectra are kept in shared memory (one buffer per component, also used for that
// component's FFT exchanges), so a thread holds one pencil in registers at a time. A block is W
// neighbouring lanes kx (W = NT / TT for about NT threads): wider tiles give longer contiguous row
// segments in B and in the Green octant, narrower ones more blocks per SM; the autotuner chooses.
// Mirrored tiles (MIR) split the W lanes into two rows of W/2: row ky and its mirror Ly - ky (0 with
// Ly/2). Both rows read the same Green octant column (|ky| is the same), so a warp loads each octant
// value once for two pencils and the octant is not fetched a second time for the mirrored row.
template <typename T, int L, int NT = 128, bool MIR = false> struct P3Cfg {
  static constexpr int TT = Plan<T, L>::TT;
  static constexpr int W0 = NT / TT;
  static constexpr int W = W0 < 1 ? 1 : (W0 > 32 ? 32 : W0);
  static constexpr int NTH = W * TT;                 // threads launched per block
  static constexpr int MINB = NTH >= 512 ? 1 : 512 / NTH;  // blocks per SM the register budget is set for
  static constexpr bool kMir = MIR && W >= 2;
  static constexpr int WH = kMir ? W / 2 : W;  // lanes per y row
  // TMA staging of the input pencils needs box rows of a multiple of 16 bytes (WH lanes per row)
  static constexpr bool kTmaOk = (WH * (int)sizeof(C<T>)) % 16 == 0;
  static constexpr int BZ = L < 256 ? L : 256;  // rows per TMA box (the box limit is 256)
  static constexpr size_t kSpecBytes = 3 * (size_t)L * W * sizeof(C<T>);
  // spectra + 3 mbarriers + room to align the spectra (and TMA destinations) to 128 bytes
  static constexpr size_t kSmem = kSpecBytes + 64 + 128;
};

// TMA: all three components' input pencils (W lanes x L positions, the zero padding and positions
// outside the source slab filled by the copy engine) are staged into the spectrum buffers by
// asynchronous tensor copies issued at kernel start, so the loads of components 1 and 2 overlap the FFT
// of component 0. Otherwise each component is loaded into registers just before its FFT. A staging
// wait that exceeds its spin limit sets *err, waits (bounded) for the other copies and ends the block.
template <typename T, int L, int NT, bool TMA, bool MIR>
__global__ void __launch_bounds__(P3Cfg<T, L, NT, MIR>::NTH, P3Cfg<T, L, NT, MIR>::MINB) k_p3_spectral(
    const C<T>* __restrict__ Bin, long in_cs, int nzs, int os, C<T>* __restrict__ Bout, long out_cs,
    int nzt, int ot, const C<T>* __restrict__ G, int Lx, int Ly, const C<T>* __restrict__ tw,
    const __grid_constant__ CUtensorMap tmap, int* __restrict__ err) {
  using Cfg = P3Cfg<T, L, NT, MIR>;
  constexpr int E = Plan<T, L>::E, TT = Plan<T, L>::TT, W = Cfg::W, WH = Cfg::WH;
  constexpr bool kTma = TMA && Cfg::kTmaOk, kMir = Cfg::kMir;
  extern __shared__ __align__(128) unsigned char p3_dyn[];
  unsigned char* sbase = p3_dyn + ((128u - (smem_addr(p3_dyn) & 127u)) & 127u);
  C<T>* spec_base = reinterpret_cast<C<T>*>(sbase);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sbase + Cfg::kSpecBytes);
  (void)bar;
  // spectrum c of the block: [row half][position][WH lanes]; this thread's column is lane l of half h
  auto spec = [spec_base](int c) { return spec_base + c * (L * W); };
  const int w = threadIdx.x, t = threadIdx.y;
  const int h = kMir ? w / WH : 0, l = kMir ? w % WH : w;
  const int ky_mirror = blockIdx.y == 0 ? Ly / 2 : Ly - (int)blockIdx.y;
  const int kx = blockIdx.x * WH + l, ky = h == 0 ? (int)blockIdx.y : ky_mirror;
  auto col = [&](int c) { return spec(c) + h * (L * WH) + l; };
  const bool act = kx < Lx;
  const long plane = (long)Ly * Lx, off = (long)ky * Lx + kx;
  C<T> v[E];
  if constexpr (kTma) {
    const int tid = t * W + w;
    if (tid == 0) {
      for (int c = 0; c < 3; ++c) mbar_init(bar + c, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
      constexpr int R = (int)sizeof(C<T>) / 8;  // 8-byte tensor elements per complex value
      for (int c = 0; c < 3; ++c) {
        mbar_expect_tx(bar + c, (unsigned)(L * W * sizeof(C<T>)));
        for (int hh = 0; hh < (kMir ? 2 : 1); ++hh)
          for (int k = 0; k < L / Cfg::BZ; ++k)
            tma_load_4d(spec(c) + (size_t)hh * L * WH + (size_t)k * Cfg::BZ * WH, &tmap, (int)blockIdx.x * WH * R,
                        hh == 0 ? (int)blockIdx.y : ky_mirror, k * Cfg::BZ - os, c, bar + c);
      }
    }
  }
  if constexpr (std::is_same<T, df>::value) {
    // forward z-FFT input of component c: false when a staging wait gave up (the block then ends)
    auto load_input = [&](int c) -> bool {
      if constexpr (kTma) {
        if (!__syncthreads_and(mbar_wait(bar + c, 0))) {
          if (t == 0 && w == 0) {
            atomicExch(err, 1);
            for (int c2 = c + 1; c2 < 3; ++c2) mbar_wait(bar + c2, 0);
          }
          return false;
        }
        // staged rows are dense; positions outside the source slab hold the copy's zero fill and are
        // not read back (half of every pencil for the usual 2n padding)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int z = t + TT * m - os;
          v[m] = (z >= 0 && z < nzs) ? col(c)[(t + TT * m) * WH] : czero<C<T>>();
        }
        __syncthreads();  // every thread holds its inputs before the exchanges overwrite spec[c]
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int z = t + TT * m - os;
          v[m] = (act && z >= 0 && z < nzs) ? Bin[c * in_cs + z * plane + off] : czero<C<T>>();
        }
      }
      return true;
    };
    // Green product at the thread's own frequencies (no other thread touches these slots).
    // The octant holds F[K_pq] for 0 <= k <= L/2 per axis; the full spectrum follows from the
    // parities of K (diagonal components even, K_pq odd along p and q): with s_a = +-1 the side of
    // axis a, F[K_pq](k) = s_p s_q F[K_pq](|k|), so Y_p = sum_q s_p s_q F_pq(|k|) J_q: the diagonal terms
    // carry no sign and the off-diagonal ones the products s_x s_y, s_x s_z, s_y s_z. Register m of a
    // pencil holds kz = t + TT*m, which lies in the lower half exactly when m < E/2 (the Nyquist
    // frequency kz = L/2, where the odd components vanish, may take either side).
    auto green_product = [&]() {
      if (!act) return;
      const int ox = Lx / 2 + 1, oy = Ly / 2 + 1;
      const long ocs = (long)(L / 2 + 1) * oy * ox, ozs = (long)oy * ox;
      const bool xlo = kx <= Lx / 2, ylo = ky <= Ly / 2;
      const int ix = xlo ? kx : Lx - kx, iy = ylo ? ky : Ly - ky;
      const bool nxy = xlo != ylo;
      const C<T>* gb = G + (long)iy * ox + ix;
      LaneSM<T, WH> s0{col(0)}, s1{col(1)}, s2{col(2)};
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const bool zlo = (E == 1) || (m < E / 2);  // lower half of kz: s_z = +1
        const int kz = t + TT * m, iz = zlo ? kz : L - kz;
        const bool nxz = zlo ? !xlo : xlo, nyz = zlo ? !ylo : ylo;
        const C<T>* g = gb + iz * ozs;
        const C<T> gxx = ldgv(g), gyy = ldgv(g + ocs), gzz = ldgv(g + 2 * ocs);
        const C<T> gxy = ldgv(g + 3 * ocs), gxz = ldgv(g + 4 * ocs), gyz = ldgv(g + 5 * ocs);
        const C<T> j0 = s0.ld(kz), j1 = s1.ld(kz), j2 = s2.ld(kz);
        s0.st(kz, add_signed(add_signed(cmul(gxx, j0), nxy, cmul(gxy, j1)), nxz, cmul(gxz, j2)));
        s1.st(kz, add_signed(add_signed(cmul(gyy, j1), nxy, cmul(gxy, j0)), nyz, cmul(gyz, j2)));
        s2.st(kz, add_signed(add_signed(cmul(gzz, j2), nxz, cmul(gxz, j0)), nyz, cmul(gyz, j1)));
      }
    };
    // the spectrum of component c back into registers, for its inverse transform
    auto load_spectrum = [&](const LaneSM<T, WH>& sm) {
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = sm.ld(t + TT * m);
      __syncthreads();  // every thread holds its inputs before the exchanges overwrite spec[c]
    };
    // crop: the target slab's positions of the inverse transform
    auto store_output = [&](int c) {
      if (!act) return;
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const int z = t + TT * m - ot;
        if (z >= 0 && z < nzt) Bout[c * out_cs + z * plane + off] = v[m];
      }
    };
    // double-float: the six transforms share one copy of the (large) unrolled FFT code, the direction
    // given at run time, so that the kernel's code fits the instruction cache; the order of the work is
    // the same as below (three forward transforms, the Green product, three inverse transforms)
#pragma unroll 1
    for (int pass = 0; pass < 6; ++pass) {
      const bool fwd = pass < 3;
      const int c = fwd ? pass : pass - 3;
      if (pass == 3) green_product();
      LaneSM<T, WH> sm{col(c)};
      if (fwd) {
        if (!load_input(c)) return;
      } else {
        load_spectrum(sm);
      }
      pencil_fft<T, L, kRuntimeSign>(v, t, sm, tw, fwd ? -1 : +1);
      if (fwd) {
#pragma unroll
        for (int m = 0; m < E; ++m) sm.st(t + TT * m, v[m]);
      } else {
        store_output(c);
      }
    }
  } else {
    // forward z-FFT of each component; spectrum left in spec[c] at the thread's own positions
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      LaneSM<T, WH> sm{col(c)};
      if constexpr (kTma) {
        if (!__syncthreads_and(mbar_wait(bar + c, 0))) {
          if (t == 0 && w == 0) {
            atomicExch(err, 1);
            for (int c2 = c + 1; c2 < 3; ++c2) mbar_wait(bar + c2, 0);
          }
          return;
        }
        // staged rows are dense; positions outside the source slab hold the copy's zero fill and are
        // not read back (half of every pencil for the usual 2n padding)
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int z = t + TT * m - os;
          v[m] = (z >= 0 && z < nzs) ? col(c)[(t + TT * m) * WH] : czero<C<T>>();
        }
        __syncthreads();  // every thread holds its inputs before the exchanges overwrite spec[c]
      } else {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int z = t + TT * m - os;
          v[m] = (act && z >= 0 && z < nzs) ? Bin[c * in_cs + z * plane + off] : czero<C<T>>();
        }
      }
      pencil_fft<T, L, -1>(v, t, sm, tw);
#pragma unroll
      for (int m = 0; m < E; ++m) sm.st(t + TT * m, v[m]);
    }
    // Green product at the thread's own frequencies (no other thread touches these slots).
    // The octant holds F[K_pq] for 0 <= k <= L/2 per axis; the full spectrum follows from the
    // parities of K (diagonal components even, K_pq odd along p and q): with s_a = +-1 the side of
    // axis a, F[K_pq](k) = s_p s_q F[K_pq](|k|), so Y_p = sum_q s_p s_q F_pq(|k|) J_q: the diagonal terms
    // carry no sign and the off-diagonal ones the products s_x s_y, s_x s_z, s_y s_z. Register m of a
    // pencil holds kz = t + TT*m, which lies in the lower half exactly when m < E/2 (the Nyquist
    // frequency kz = L/2, where the odd components vanish, may take either side).
    if (act) {
      const int ox = Lx / 2 + 1, oy = Ly / 2 + 1;
      const long ocs = (long)(L / 2 + 1) * oy * ox, ozs = (long)oy * ox;
      const bool xlo = kx <= Lx / 2, ylo = ky <= Ly / 2;
      const int ix = xlo ? kx : Lx - kx, iy = ylo ? ky : Ly - ky;
      const bool nxy = xlo != ylo;
      const C<T>* gb = G + (long)iy * ox + ix;
      LaneSM<T, WH> s0{col(0)}, s1{col(1)}, s2{col(2)};
#pragma unroll
      for (int m = 0; m < E; ++m) {
        const bool zlo = (E == 1) || (m < E / 2);  // lower half of kz: s_z = +1
        const int kz = t + TT * m, iz = zlo ? kz : L - kz;
        const bool nxz = zlo ? !xlo : xlo, nyz = zlo ? !ylo : ylo;
        const C<T>* g = gb + iz * ozs;
        const C<T> gxx = ldgv(g), gyy = ldgv(g + ocs), gzz = ldgv(g + 2 * ocs);
        const C<T> gxy = ldgv(g + 3 * ocs), gxz = ldgv(g + 4 * ocs), gyz = ldgv(g + 5 * ocs);
        const C<T> j0 = s0.ld(kz), j1 = s1.ld(kz), j2 = s2.ld(kz);
        s0.st(kz, add_signed(add_signed(cmul(gxx, j0), nxy, cmul(gxy, j1)), nxz, cmul(gxz, j2)));
        s1.st(kz, add_signed(add_signed(cmul(gyy, j1), nxy, cmul(gxy, j0)), nyz, cmul(gyz, j2)));
        s2.st(kz, add_signed(add_signed(cmul(gzz, j2), nxz, cmul(gxz, j0)), nyz, cmul(gyz, j1)));
      }
    }
    // inverse z-FFT of each component and crop
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      LaneSM<T, WH> sm{col(c)};
#pragma unroll
      for (int m = 0; m < E; ++m) v[m] = sm.ld(t + TT * m);
      __syncthreads();  // every thread holds its inputs before the exchanges overwrite spec[c]
      pencil_fft<T, L, +1>(v, t, sm, tw);
      if (act) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
          const int z = t + TT * m - ot;
          if (z >= 0 && z < nzt) Bout[c * out_cs + z * plane + off] = v[m];
        }
      }
    }
  }
}

// ---------------------------------------------------------------- contiguous full FFT (setup)
template <typename T, int L, int SIGN>
__global__ void __launch_bounds__(kThreads) k_rows_fft(C<T>* __restrict__ data, long nrows,
                                                      const C<T>* __restrict__ tw) {
  constexpr int E = Plan<T, L>::E, TT = Plan<T, L>::TT, P = RowCfg<T, L>::P;
  __shared__ C<T> smem[P * RowSM<T>::words(L)];
  const int t = threadIdx.x, p = threadIdx.y;
  const long row = (long)blockIdx.x * P + p;
  const bool act = row < nrows;
  RowSM<T> sm{smem + p * RowSM<T>::words(L)};
  C<T> v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = act ? data[row * L + t + TT * m] : czero<C<T>>();
  pencil_fft<T, L, SIGN>(v, t, sm, tw);
  if (act) {
#pragma unroll
    for (int m = 0; m < E; ++m) data[row * L + t + TT * m] = v[m];
  }
}

}  // namespace ie
