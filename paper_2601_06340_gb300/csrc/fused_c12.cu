#include "fused_launch.cuh"
BPM_INSTANTIATE_FUSED3(12)
