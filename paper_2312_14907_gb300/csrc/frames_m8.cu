// frames_m8.cu -- the fused frame kernel instantiated for M = 8.
#include "frames_inst.cuh"

MPBP_DEFINE_FRAMES(8)
