// The multigrid CG launches of 3D problems with FP32 CG vectors (explicit instances).
#include "fo_mg.cuh"

FO_MG_DEFINE(3, 1, true, 1, float)
FO_MG_DEFINE(3, 3, true, 1, float)
