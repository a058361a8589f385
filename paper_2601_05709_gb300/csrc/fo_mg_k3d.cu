// The multigrid CG launches of 3D state problems with FP64 CG vectors (explicit instances).
#include "fo_mg.cuh"

FO_MG_DEFINE(3, 1, true, 1, double)
FO_MG_DEFINE(3, 3, true, 1, double)
