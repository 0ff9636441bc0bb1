// frames_m64.cu -- the fused frame kernel instantiated for M = 64.
#include "frames_inst.cuh"

MPBP_DEFINE_FRAMES(64)
