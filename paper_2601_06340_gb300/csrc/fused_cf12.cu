#include "fused_launch.cuh"
BPM_INSTANTIATE_FUSED3F(12)
