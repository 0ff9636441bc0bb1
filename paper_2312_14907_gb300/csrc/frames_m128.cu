// frames_m128.cu -- the fused frame kernel instantiated for M = 128.
#include "frames_inst.cuh"

MPBP_DEFINE_FRAMES(128)
