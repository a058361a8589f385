// The multigrid CG launches of 2D problems with FP32 CG vectors (explicit instances).
#include "fo_mg.cuh"

FO_MG_DEFINE(2, 1, true, 1, float)
FO_MG_DEFINE(2, 2, true, 1, float)
