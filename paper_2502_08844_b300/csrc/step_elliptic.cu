// The step kernels compiled with the elliptic friction cone (used for batches that contain an
// elliptic-cone model; see step_kernels.cuh).
#define PG_WITH_ELLIPTIC 1
#define PG_STEP_NS elliptic
#include "step_kernels.cuh"
