// double instantiation of the z-pass launcher (P3), compiled apart from the other passes.
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<double>::p3(int, int, const C<double>*, long, int, int, C<double>*, long, int, int,
                                       const C<double>*, int, int, const C<double>*, int*, cudaStream_t);
}  // namespace ie
