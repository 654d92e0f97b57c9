// Temporally blocked FGP kernels (the implementation is sci_fused.cuh),
// instantiated for float storage, plus the tile-class queries.
#define SCI_FUSED_COMMON
#define SCI_FUSED_STORAGE float
#include "sci_fused.cuh"
