// Explicit instantiation of the DKSS_MUL launchers for one (m, L) pair,
// selected with -DDKSS_INST_M=<m> -DDKSS_INST_L=<L> by the build.
#include "launch.cuh"

DKSS_INSTANTIATE(DKSS_INST_M, DKSS_INST_L)
