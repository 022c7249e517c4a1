// float instantiation of the z-pass launcher (P3: z-FFT, Green product, inverse), compiled apart from
// the other float passes so the two halves build in parallel.
#include "conv_launch.cuh"
namespace ie {
template cudaError_t ConvLaunch<float>::p3(int, int, const C<float>*, long, int, int, C<float>*, long, int, int,
                                           const C<float>*, int, int, const C<float>*, int*, cudaStream_t);
}  // namespace ie
