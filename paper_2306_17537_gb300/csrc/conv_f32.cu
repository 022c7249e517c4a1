// float instantiation of the convolution pass launchers.
#include "conv_launch.cuh"
namespace ie {
template struct ConvLaunch<float>;
bool supported_pencil(int L) { return supported_pencil_impl(L); }
}  // namespace ie
