#include "fused_launch.cuh"
BPM_INSTANTIATE_FUSED4F
