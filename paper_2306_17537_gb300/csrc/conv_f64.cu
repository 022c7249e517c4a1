// double instantiation of the convolution pass launchers (the z pass in conv_f64_p3.cu).
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<double>::p1(int, const FieldC<double>*, long, const FieldR<double>*, long, C<double>*, long, int,
                                       long, const C<double>*, cudaStream_t, const FieldR<double>*, FieldC<double>*, long);
template cudaError_t ConvLaunch<double>::p5(int, int, const C<double>*, long, int, long, const FieldC<double>*, long,
                                       FieldC<double>*, long, double2*, long, const double2*, long, const C<double>*,
                                       cudaStream_t);
template cudaError_t ConvLaunch<double>::lanes(int, int, int, const C<double>*, long, long, long, int, C<double>*, long, long,
                                          long, int, int, int, int, const C<double>*, cudaStream_t);
template cudaError_t ConvLaunch<double>::rows(int, int, C<double>*, long, const C<double>*, cudaStream_t);
}  // namespace ie
