// Host-side launchers for the convolution passes: map a runtime pencil length to the kernel
// template instantiated for it. Explicitly instantiated for float and double in conv_f32.cu and
// conv_f64.cu so the two precisions compile in parallel.
#pragma once
#include "conv.cuh"
#include "conv_kernels.cuh"

#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <type_traits>

namespace ie {

#define IE_FOR_EACH_L(X) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

inline bool supported_pencil_impl(int L) {
  switch (L) {
#define IE_CASE(N) case N:
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    return true;
    default:
      return false;
  }
}


template <typename T>
cudaError_t ConvLaunch<T>::p1(int L, const FieldC<T>* x, long x_cs, const FieldR<T>* ds, long d_cs, C<T>* A,
                              long A_cs, int nx, long nrows, const C<T>* tw, cudaStream_t s, const FieldR<T>* mt,
                              FieldC<T>* w, long w_cs) {
  if (nrows <= 0) return cudaSuccess;
  if (mt && std::is_same<T, df>::value) return cudaErrorInvalidValue;  // contraction: float and double only
  switch (L) {
#define IE_CASE(N)                                                                                   \
  case N: {                                                                                          \
    constexpr int P = RowCfg<T, N>::P;                                                               \
    dim3 blk(Plan<T, N>::TT, P), grd((unsigned)((nrows + P - 1) / P));                              \
    if constexpr (!std::is_same<T, df>::value) {                                                     \
      if (mt) {                                                                                      \
        k_p1_contrast_fftx<T, N, true><<<grd, blk, 0, s>>>(x, x_cs, ds, d_cs, A, A_cs, nx, nrows, tw, mt, \
                                                           w, w_cs);                                 \
        break;                                                                                       \
      }                                                                                              \
    }                                                                                                \
    k_p1_contrast_fftx<T, N, false><<<grd, blk, 0, s>>>(x, x_cs, ds, d_cs, A, A_cs, nx, nrows, tw, nullptr, \
                                                        nullptr, 0);                                 \
    break;                                                                                           \
  }
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t ConvLaunch<T>::p5(int L, int mode, const C<T>* A, long A_cs, int nx, long nrows,
                              const FieldC<T>* xin, long x_cs, FieldC<T>* y, long y_cs, double2* r, long r_cs,
                              const double2* b, long b_cs, const C<T>* tw, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (L) {
#define IE_CASE(N)                                                                                               \
  case N: {                                                                                                      \
    constexpr int P = RowCfg<T, N>::P;                                                                           \
    dim3 blk(Plan<T, N>::TT, P), grd((unsigned)((nrows + P - 1) / P), 3);                                       \
    switch (mode) {                                                                                              \
      case EPI_APPLY:                                                                                            \
        k_p5_ifftx_epilogue<T, N, EPI_APPLY><<<grd, blk, 0, s>>>(A, A_cs, nx, nrows, xin, x_cs, y, y_cs, r,     \
                                                                 r_cs, b, b_cs, tw);                             \
        break;                                                                                                   \
      case EPI_CONV:                                                                                             \
        k_p5_ifftx_epilogue<T, N, EPI_CONV><<<grd, blk, 0, s>>>(A, A_cs, nx, nrows, xin, x_cs, y, y_cs, r,      \
                                                                r_cs, b, b_cs, tw);                              \
        break;                                                                                                   \
      case EPI_ACCUM128:                                                                                         \
        k_p5_ifftx_epilogue<T, N, EPI_ACCUM128><<<grd, blk, 0, s>>>(A, A_cs, nx, nrows, xin, x_cs, y, y_cs, r,  \
                                                                    r_cs, b, b_cs, tw);                          \
        break;                                                                                                   \
      case EPI_RESID128:                                                                                         \
        k_p5_ifftx_epilogue<T, N, EPI_RESID128><<<grd, blk, 0, s>>>(A, A_cs, nx, nrows, xin, x_cs, y, y_cs, r,  \
                                                                    r_cs, b, b_cs, tw);                          \
        break;                                                                                                   \
      default:                                                                                                   \
        return cudaErrorInvalidValue;                                                                            \
    }                                                                                                            \
    break;                                                                                                       \
  }
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T, int N, int NT>
static cudaError_t lanes_launch(int sign, const C<T>* in, long in_cs, long in_zs, long in_es, int n_in, C<T>* out,
                                long out_cs, long out_zs, long out_es, int n_out, int nlanes, int nbatch, int ncomp,
                                const C<T>* tw, cudaStream_t s) {
  using Cfg = LaneCfg<T, N, NT>;
  constexpr int W = Cfg::W;
  static std::once_flag attr;
  static cudaError_t ae = cudaSuccess;
  std::call_once(attr, [] {
    if (Cfg::kSmem > 48 * 1024) {
      ae = cudaFuncSetAttribute(k_lanes_fft<T, N, -1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
      if (ae == cudaSuccess)
        ae = cudaFuncSetAttribute(k_lanes_fft<T, N, 1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::kSmem);
    }
  });
  if (ae != cudaSuccess) return ae;
  dim3 blk(W, Plan<T, N>::TT), grd((unsigned)((nlanes + W - 1) / W), (unsigned)nbatch, (unsigned)ncomp);
  if (sign < 0)
    k_lanes_fft<T, N, -1, NT><<<grd, blk, Cfg::kSmem, s>>>(in, in_cs, in_zs, in_es, n_in, out, out_cs, out_zs, out_es,
                                                            n_out, nlanes, tw);
  else
    k_lanes_fft<T, N, 1, NT><<<grd, blk, Cfg::kSmem, s>>>(in, in_cs, in_zs, in_es, n_in, out, out_cs, out_zs, out_es,
                                                           n_out, nlanes, tw);
  return cudaGetLastError();
}

template <typename T>
cudaError_t ConvLaunch<T>::lanes(int L, int sign, int variant, const C<T>* in, long in_cs, long in_zs, long in_es,
                                 int n_in, C<T>* out, long out_cs, long out_zs, long out_es, int n_out, int nlanes,
                                 int nbatch, int ncomp, const C<T>* tw, cudaStream_t s) {
  if (nbatch <= 0 || nlanes <= 0 || ncomp <= 0) return cudaSuccess;
  switch (L) {
#define IE_CASE(N)                                                                                                  \
  case N:                                                                                                           \
    switch (variant) {                                                                                              \
      case 1: return lanes_launch<T, N, 128>(sign, in, in_cs, in_zs, in_es, n_in, out, out_cs, out_zs, out_es, n_out, \
                                             nlanes, nbatch, ncomp, tw, s);                                          \
      case 2: return lanes_launch<T, N, 512>(sign, in, in_cs, in_zs, in_es, n_in, out, out_cs, out_zs, out_es, n_out, \
                                             nlanes, nbatch, ncomp, tw, s);                                          \
      default: return lanes_launch<T, N, 256>(sign, in, in_cs, in_zs, in_es, n_in, out, out_cs, out_zs, out_es, n_out,\
                                              nlanes, nbatch, ncomp, tw, s);                                         \
    }
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

// cuTensorMapEncodeTiled from the CUDA driver, looked up once (null when the CUDA driver lacks it).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// TMA = true stages the input pencils with tensor copies when the tile allows it (P3Cfg::kTmaOk) and
// the CUDA driver provides the tensor-map encoder; otherwise the same tile runs with register loads.
// MIR = true pairs each row ky with its mirror (P3Cfg::kMir; a one-lane tile runs unpaired).
// Every tile keeps its spectra in dynamic shared memory (above the 48 KB default for the wider tiles).
template <typename T, int N, int NT, bool TMA, bool MIR>
static cudaError_t p3_run(const C<T>* Bin, long in_cs, int nzs, int os, C<T>* Bout, long out_cs, int nzt, int ot,
                          const C<T>* G, int Lx, int Ly, const C<T>* tw, int* err, const CUtensorMap& map,
                          cudaStream_t s) {
  using Cfg = P3Cfg<T, N, NT, MIR>;
  static std::once_flag attr;
  static cudaError_t ae = cudaSuccess;
  std::call_once(attr, [] {
    if (Cfg::kSmem > 48 * 1024)
      ae = cudaFuncSetAttribute(k_p3_spectral<T, N, NT, TMA, MIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg::kSmem);
  });
  if (ae != cudaSuccess) return ae;
  const unsigned gy = Cfg::kMir ? (unsigned)(Ly / 2) : (unsigned)Ly;
  dim3 blk(Cfg::W, Plan<T, N>::TT), grd((unsigned)((Lx + Cfg::WH - 1) / Cfg::WH), gy);
  k_p3_spectral<T, N, NT, TMA, MIR><<<grd, blk, Cfg::kSmem, s>>>(Bin, in_cs, nzs, os, Bout, out_cs, nzt, ot, G, Lx,
                                                                 Ly, tw, map, err);
  return cudaGetLastError();
}

template <typename T, int N, int NT, bool TMA, bool MIR = false>
static cudaError_t p3_launch(const C<T>* Bin, long in_cs, int nzs, int os, C<T>* Bout, long out_cs, int nzt, int ot,
                             const C<T>* G, int Lx, int Ly, const C<T>* tw, int* err, cudaStream_t s) {
  using Cfg = P3Cfg<T, N, NT, MIR>;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  if (Cfg::kMir && Ly % 2 != 0) return cudaErrorInvalidValue;  // padded lengths are even
  if constexpr (TMA && Cfg::kTmaOk) {
    auto enc = tensor_map_encoder();
    if (enc) {
      // B viewed as 8-byte elements: (x = Lx * R, y = Ly, z = nzs source rows, component)
      constexpr int R = (int)sizeof(C<T>) / 8;
      const cuuint64_t dims[4] = {(cuuint64_t)Lx * R, (cuuint64_t)Ly, (cuuint64_t)nzs, 3};
      const cuuint64_t strides[3] = {(cuuint64_t)Lx * R * 8, (cuuint64_t)Ly * Lx * R * 8, (cuuint64_t)in_cs * R * 8};
      const cuuint32_t box[4] = {(cuuint32_t)(Cfg::WH * R), 1, (cuuint32_t)Cfg::BZ, 1};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<C<T>*>(Bin), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
      return p3_run<T, N, NT, true, MIR>(Bin, in_cs, nzs, os, Bout, out_cs, nzt, ot, G, Lx, Ly, tw, err, map, s);
    }
  }
  return p3_run<T, N, NT, false, MIR>(Bin, in_cs, nzs, os, Bout, out_cs, nzt, ot, G, Lx, Ly, tw, err, map, s);
}

// The mirrored 256-thread tiles (variants 8, 9) are built for float only: the complex64 operator runs
// on sub-domains of every shape, the complex128 and double-float ones mostly on the whole grid, where
// the 512-thread tiles win, and each further instantiation lengthens the build of those units.
template <typename T> constexpr bool kMir256 = std::is_same<T, float>::value;

template <typename T>
cudaError_t ConvLaunch<T>::p3(int L, int variant, const C<T>* Bin, long in_cs, int nzs, int os, C<T>* Bout,
                              long out_cs, int nzt, int ot, const C<T>* G, int Lx, int Ly, const C<T>* tw, int* err,
                              cudaStream_t s) {
#define IE_P3(N, NT, TMA, MIR) \
  p3_launch<T, N, NT, TMA, MIR>(Bin, in_cs, nzs, os, Bout, out_cs, nzt, ot, G, Lx, Ly, tw, err, s)
  switch (L) {
#define IE_CASE(N)                                                                  \
  case N:                                                                           \
    switch (variant) {                                                              \
      case 1: return IE_P3(N, 64, false, false);                                    \
      case 2: return IE_P3(N, 128, true, false);                                    \
      case 3: return IE_P3(N, 64, true, false);                                     \
      case 4: return IE_P3(N, 256, false, false);                                   \
      case 5: return IE_P3(N, 256, true, false);                                    \
      case 6: return IE_P3(N, 512, false, false);                                   \
      case 7: return IE_P3(N, 512, true, false);                                    \
      case 8:                                                                       \
        if constexpr (kMir256<T>) return IE_P3(N, 256, false, true);                \
        else return cudaErrorNotSupported;                                          \
      case 9:                                                                       \
        if constexpr (kMir256<T>) return IE_P3(N, 256, true, true);                 \
        else return cudaErrorNotSupported;                                          \
      case 10: return IE_P3(N, 512, false, true);                                   \
      case 11: return IE_P3(N, 512, true, true);                                    \
      default: return IE_P3(N, 128, false, false);                                  \
    }
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    default:
      return cudaErrorInvalidValue;
  }
#undef IE_P3
}

template <typename T>
cudaError_t ConvLaunch<T>::rows(int L, int sign, C<T>* data, long nrows, const C<T>* tw, cudaStream_t s) {
  if (nrows <= 0) return cudaSuccess;
  switch (L) {
#define IE_CASE(N)                                                                    \
  case N: {                                                                           \
    constexpr int P = RowCfg<T, N>::P;                                                \
    dim3 blk(Plan<T, N>::TT, P), grd((unsigned)((nrows + P - 1) / P));               \
    if (sign < 0)                                                                     \
      k_rows_fft<T, N, -1><<<grd, blk, 0, s>>>(data, nrows, tw);                      \
    else                                                                              \
      k_rows_fft<T, N, 1><<<grd, blk, 0, s>>>(data, nrows, tw);                       \
    break;                                                                            \
  }
    IE_FOR_EACH_L(IE_CASE)
#undef IE_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ie
