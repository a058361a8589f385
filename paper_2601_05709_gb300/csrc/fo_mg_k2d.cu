// The multigrid CG launches of 2D problems with FP64 CG vectors (explicit instances).
#include "fo_mg.cuh"

FO_MG_DEFINE(2, 1, true, 1, double)
FO_MG_DEFINE(2, 2, true, 1, double)
FO_MG_DEFINE(2, 2, false, 2, double)
