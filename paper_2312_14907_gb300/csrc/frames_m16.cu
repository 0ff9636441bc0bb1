// frames_m16.cu -- the fused frame kernel instantiated for M = 16.
#include "frames_inst.cuh"

MPBP_DEFINE_FRAMES(16)
