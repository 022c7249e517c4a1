// float instantiation of the convolution pass launchers (the z pass, the largest, in conv_f32_p3.cu).
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<float>::p1(int, const FieldC<float>*, long, const FieldR<float>*, long, C<float>*,
                                           long, int, long, const C<float>*, cudaStream_t, const FieldR<float>*,
                                           FieldC<float>*, long);
template cudaError_t ConvLaunch<float>::p5(int, int, const C<float>*, long, int, long, const FieldC<float>*, long,
                                           FieldC<float>*, long, double2*, long, const double2*, long,
                                           const C<float>*, cudaStream_t);
template cudaError_t ConvLaunch<float>::lanes(int, int, int, const C<float>*, long, long, long, int, C<float>*, long,
                                              long, long, int, int, int, int, const C<float>*, cudaStream_t);
template cudaError_t ConvLaunch<float>::rows(int, int, C<float>*, long, const C<float>*, cudaStream_t);
bool supported_pencil(int L) { return supported_pencil_impl(L); }
}  // namespace ie
