// frames_m32.cu -- the fused frame kernel instantiated for M = 32.
#include "frames_inst.cuh"

MPBP_DEFINE_FRAMES(32)
