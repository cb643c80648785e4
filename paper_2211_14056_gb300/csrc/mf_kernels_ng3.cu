// Kernels for gg -> t tbar + 1 gluon(s): 3 gluons in the colour-ordered recursion.
#include "mf_kernels.cuh"
MF_INSTANTIATE(3)
