// Explicit instantiation of the DKSS_MUL launchers for one (m, L, LR) triple
// (ring degree m, 32-bit limbs L of stored residues, 26-bit limbs LR of the
// product arithmetic), selected with -DDKSS_INST_M/-DDKSS_INST_L/-DDKSS_INST_LR.
#include "launch.cuh"

DKSS_INSTANTIATE(DKSS_INST_M, DKSS_INST_L, DKSS_INST_LR)
