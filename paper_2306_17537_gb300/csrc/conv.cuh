// Declarations of the convolution pass launchers (definitions in conv_launch.cuh, instantiated
// for float in conv_f32.cu and for double in conv_f64.cu).
#pragma once
#include "common.cuh"

namespace ie {

enum Epilogue { EPI_APPLY = 0, EPI_ACCUM128 = 1, EPI_RESID128 = 2, EPI_CONV = 3 };

bool supported_pencil(int L);
constexpr int kTileVariants = 3;    // P2, P4
constexpr int kP3TileVariants = 12;  // P3 (see ConvLaunch::p3)

template <typename T> struct ConvLaunch {
  // mt != nullptr: contraction form (ds = dsigma M, mt = M); also stores w = M x at stride w_cs
  static cudaError_t p1(int L, const FieldC<T>* x, long x_cs, const FieldR<T>* ds, long d_cs, C<T>* A, long A_cs,
                        int nx, long nrows, const C<T>* tw, cudaStream_t s, const FieldR<T>* mt = nullptr,
                        FieldC<T>* w = nullptr, long w_cs = 0);
  static cudaError_t p5(int L, int mode, const C<T>* A, long A_cs, int nx, long nrows, const FieldC<T>* xin,
                        long x_cs, FieldC<T>* y, long y_cs, double2* r, long r_cs, const double2* b, long b_cs,
                        const C<T>* tw, cudaStream_t s);
  // variant: tiles of about 256 (0), 128 (1) and 512 (2) threads (choices for the autotuner)
  static cudaError_t lanes(int L, int sign, int variant, const C<T>* in, long in_cs, long in_zs, long in_es,
                           int n_in, C<T>* out, long out_cs, long out_zs, long out_es, int n_out, int nlanes,
                           int nbatch, int ncomp, const C<T>* tw, cudaStream_t s);
  // variant: tiles of about 128 (0), 64 (1), 256 (4) and 512 (6) threads, and the same with TMA staging
  // of the input pencils (2, 3, 5, 7); 256 and 512 threads with mirrored rows ky, Ly - ky (8, 10) and
  // the same with TMA staging (9, 11). Variants 8 and 9 exist for float only: for the other types
  // they return cudaErrorNotSupported without launching (the autotuner skips them);
  // err: set to 1 (device) if a staging wait of a TMA variant gave up
  static cudaError_t p3(int L, int variant, const C<T>* Bin, long in_cs, int nzs, int os, C<T>* Bout, long out_cs,
                        int nzt, int ot, const C<T>* G, int Lx, int Ly, const C<T>* tw, int* err, cudaStream_t s);
  static cudaError_t rows(int L, int sign, C<T>* data, long nrows, const C<T>* tw, cudaStream_t s);
};
extern template struct ConvLaunch<float>;
extern template struct ConvLaunch<double>;
extern template struct ConvLaunch<df>;

}  // namespace ie
