// The multigrid CG launch of the 3D velocity form (three component systems; explicit instance).
#include "fo_mg.cuh"

FO_MG_DEFINE(3, 3, false, 3, double)
