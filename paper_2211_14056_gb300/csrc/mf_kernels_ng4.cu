// Kernels for gg -> t tbar + 2 gluon(s): 4 gluons in the colour-ordered recursion.
#include "mf_kernels.cuh"
MF_INSTANTIATE(4)
