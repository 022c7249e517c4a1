// double-float instantiation of the convolution pass launchers (the z pass in conv_df_p3.cu).
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<df>::p1(int, const FieldC<df>*, long, const FieldR<df>*, long, C<df>*, long, int,
                                       long, const C<df>*, cudaStream_t, const FieldR<df>*, FieldC<df>*, long);
template cudaError_t ConvLaunch<df>::p5(int, int, const C<df>*, long, int, long, const FieldC<df>*, long,
                                       FieldC<df>*, long, double2*, long, const double2*, long, const C<df>*,
                                       cudaStream_t);
template cudaError_t ConvLaunch<df>::lanes(int, int, int, const C<df>*, long, long, long, int, C<df>*, long, long,
                                          long, int, int, int, int, const C<df>*, cudaStream_t);
template cudaError_t ConvLaunch<df>::rows(int, int, C<df>*, long, const C<df>*, cudaStream_t);
}  // namespace ie
