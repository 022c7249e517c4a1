// Register-resident radix-16/8 Stockham FFT on one pencil, exchanged through shared memory.
//
// A pencil of length L (a power of two, 2..1024) is owned by TT = L/E threads; thread t holds the
// E elements t + TT*m (m = 0..E-1) in registers on entry and on exit, in natural order. Stage s
// (radix R_s, stride Ns = R_0*...*R_{s-1}) treats butterfly j with inputs j + r*L/R_s, multiplies
// input r by exp(sign*2*pi*i*(j mod Ns)*r/(Ns*R_s)), applies an R_s-point DFT and writes output r to
// position (j - j mod Ns)*R_s + (j mod Ns) + r*Ns (Stockham autosort: natural order after the last
// stage, no bit reversal). Between stages the data goes through shared memory; the first stage reads
// registers and the last stage writes registers, so a pencil of length E needs no shared memory and
// a forward transform can be followed by pointwise work and the inverse transform in registers.
//
// E = 16 for float and 8 for double and double-float (register budget), so L = 256 in float is two
// radix-16 stages with a single shared-memory exchange.
#pragma once
#include "common.cuh"

namespace ie {

template <typename T> struct EMax;
template <> struct EMax<float> { static constexpr int v = 16; };
template <> struct EMax<double> { static constexpr int v = 8; };
template <> struct EMax<df> { static constexpr int v = 8; };

template <typename T, int L> struct Plan {
  static constexpr int E = L < EMax<T>::v ? L : EMax<T>::v;  // elements per thread
  static constexpr int TT = L / E;                           // threads per pencil
};

// SIGN = -1 (forward) or +1 (inverse) fixes the direction at compile time; SIGN = 0 takes it from the
// run-time argument sgn instead, so that one copy of the code serves both directions (used where the
// unrolled transforms are large enough to miss the instruction cache).
constexpr int kRuntimeSign = 0;

// x * exp(s * 2 pi i q / 16), q in [0, 8), s = SIGN (or sgn), with the trivial rotations done without
// multiplies.
template <typename T, int SIGN> __device__ __forceinline__ C<T> rot16(int q, C<T> x, int sgn = SIGN) {
  const int sg = SIGN != 0 ? SIGN : sgn;
  constexpr T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
  if (q == 0) return x;
  if (q == 4) return sg < 0 ? mk<T>(x.y, -x.x) : mk<T>(-x.y, x.x);
  T wr, wi;
  switch (q) {
    case 1: wr = c1; wi = s1; break;
    case 2: wr = h; wi = h; break;
    case 3: wr = s1; wi = c1; break;
    case 5: wr = -s1; wi = c1; break;
    case 6: wr = -h; wi = h; break;
    default: wr = -c1; wi = s1; break;  // q == 7
  }
  return cmul(x, mk<T>(wr, sg < 0 ? -wi : wi));
}

// In-place R-point DFT (R <= 16) on natural-order registers, radix-2 decimation in time.
template <typename T, int R, int SIGN> struct DFT {
  __device__ __forceinline__ static void run(C<T>* v, int sgn = SIGN) {
    C<T> e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) {
      e[i] = v[2 * i];
      o[i] = v[2 * i + 1];
    }
    DFT<T, R / 2, SIGN>::run(e, sgn);
    DFT<T, R / 2, SIGN>::run(o, sgn);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      C<T> t = rot16<T, SIGN>(k * (16 / R), o[k], sgn);
      v[k] = e[k] + t;
      v[k + R / 2] = e[k] - t;
    }
  }
};
template <typename T, int SIGN> struct DFT<T, 1, SIGN> {
  __device__ __forceinline__ static void run(C<T>*, int = SIGN) {}
};
template <typename T, int SIGN> struct DFT<T, 2, SIGN> {
  __device__ __forceinline__ static void run(C<T>* v, int = SIGN) {
    C<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  }
};

// Shared-memory views of one pencil.
// Contiguous pencils (one per row): one padding slot per 16 elements keeps stage writes
// conflict-free.
template <typename T> struct RowSM {
  C<T>* base;
  __device__ __forceinline__ C<T> ld(int i) const { return base[i + (i >> 4)]; }
  __device__ __forceinline__ void st(int i, C<T> x) const { base[i + (i >> 4)] = x; }
  __host__ __device__ static constexpr int words(int L) { return L + L / 16; }
};
// W side-by-side pencils (lanes contiguous in memory): element i of lane w at [i][w]. When a row of W
// elements is narrower than a 128-byte bank line (RPL rows per line), row i is stored at i XOR
// ((i / 16) mod RPL): the first stage writes rows 16 apart from neighbouring threads of a warp, and
// the XOR spreads them over the line (a permutation inside each aligned group of 16 rows, so runs of
// consecutive rows stay on distinct banks).
template <typename T, int W> struct LaneSM {
  C<T>* base;  // already offset by the lane
  static constexpr int kRowBytes = W * (int)sizeof(C<T>);
  static constexpr int RPL = kRowBytes < 128 ? 128 / kRowBytes : 1;
  __device__ __forceinline__ int row(int i) const { return RPL > 1 ? (i ^ ((i >> 4) & (RPL - 1))) : i; }
  __device__ __forceinline__ C<T> ld(int i) const { return base[row(i) * W]; }
  __device__ __forceinline__ void st(int i, C<T> x) const { base[row(i) * W] = x; }
};

template <typename T, int SIGN>
__device__ __forceinline__ C<T> twiddle(const C<T>* __restrict__ tw, int idx, int sgn = SIGN) {
  C<T> w = ldgv(tw + idx);
  if ((SIGN != 0 ? SIGN : sgn) > 0) w.y = -w.y;
  return w;
}

// Butterfly twiddles p[r] = w^r (r = 1..R-1), w = exp(SIGN 2 pi i q / TWN) for the table index q of r = 1.
// In float only the power-of-two entries w, w^2, w^4, w^8 are loaded and the others formed as products
// of those (r's binary digits): at most four rounded table entries and three roundings per twiddle, a
// few float ulps, and a third to a quarter of the table loads, which share the load/store pipe with the
// shared-memory exchanges. In double and double-float every twiddle is a table entry.
template <typename T> struct TwiddlePowers { static constexpr bool v = false; };
template <> struct TwiddlePowers<float> { static constexpr bool v = true; };

template <typename T, int R, int SIGN>
__device__ __forceinline__ void butterfly_twiddles(const C<T>* __restrict__ tw, int q, C<T> (&p)[R],
                                                   int sgn = SIGN) {
  if constexpr (TwiddlePowers<T>::v) {
#pragma unroll
    for (int b = 1; b < R; b <<= 1) p[b] = twiddle<T, SIGN>(tw, q * b, sgn);
#pragma unroll
    for (int r = 3; r < R; ++r) {
      if (r & (r - 1)) {
        int hb = r;
        while (hb & (hb - 1)) hb &= hb - 1;  // highest power of two in r
        p[r] = cmul(p[hb], p[r - hb]);
      }
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) p[r] = twiddle<T, SIGN>(tw, q * r, sgn);
  }
}

template <typename T, int L, int SIGN, int NS, class SM> struct Stages {
  static constexpr int E = Plan<T, L>::E;
  static constexpr int TT = Plan<T, L>::TT;
  static constexpr int REM = L / NS;
  static constexpr int R = REM < E ? REM : E;
  static constexpr int NB = E / R;
  static constexpr bool FIRST = (NS == 1);
  static constexpr bool LAST = (NS * R == L);

  __device__ __forceinline__ static void run(C<T> (&v)[E], int t, const SM& sm, const C<T>* __restrict__ tw,
                                             int sgn = SIGN) {
    C<T> x[NB][R];
    if constexpr (FIRST) {
#pragma unroll
      for (int r = 0; r < R; ++r) x[0][r] = v[r];
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) x[b][r] = sm.ld(t + TT * b + r * (L / R));
      __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if constexpr (!FIRST) {
        const int j = t + TT * b;
        const int k = j & (NS - 1);
        C<T> p[R];
        butterfly_twiddles<T, R, SIGN>(tw, k * (TWN / (NS * R)), p, sgn);
#pragma unroll
        for (int r = 1; r < R; ++r) x[b][r] = cmul(x[b][r], p[r]);
      }
      DFT<T, R, SIGN>::run(x[b], sgn);
    }
    if constexpr (LAST) {
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) v[b + r * NB] = x[b][r];
    } else {
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = t + TT * b;
        const int k = j & (NS - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) sm.st(base + r * NS, x[b][r]);
      }
      __syncthreads();
      Stages<T, L, SIGN, (LAST ? NS : NS * R), SM>::run(v, t, sm, tw, sgn);
    }
  }
};

// Forward (SIGN = -1) or unnormalised inverse (SIGN = +1) DFT of one pencil held as described above;
// SIGN = kRuntimeSign takes the direction from sgn. Every thread of the block must call it (it contains
// __syncthreads when L > E).
template <typename T, int L, int SIGN, class SM>
__device__ __forceinline__ void pencil_fft(C<T> (&v)[Plan<T, L>::E], int t, const SM& sm,
                                           const C<T>* __restrict__ tw, int sgn = SIGN) {
  Stages<T, L, SIGN, 1, SM>::run(v, t, sm, tw, sgn);
}

}  // namespace ie
