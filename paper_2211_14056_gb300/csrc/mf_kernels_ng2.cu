// Kernels for gg -> t tbar + 0 gluon(s): 2 gluons in the colour-ordered recursion.
#include "mf_kernels.cuh"
MF_INSTANTIATE(2)
