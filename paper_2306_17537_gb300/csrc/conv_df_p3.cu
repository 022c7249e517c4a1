// double-float instantiation of the z-pass launcher (P3), compiled apart from the other passes.
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<df>::p3(int, int, const C<df>*, long, int, int, C<df>*, long, int, int,
                                       const C<df>*, int, int, const C<df>*, int*, cudaStream_t);
}  // namespace ie
