// double instantiation of the convolution pass launchers.
#include "conv_launch.cuh"
namespace ie { template struct ConvLaunch<double>; }
