// double-float instantiation of the convolution pass launchers (FP64-accurate residual).
#include "conv_launch.cuh"
namespace ie {
template struct ConvLaunch<df>;
}  // namespace ie
