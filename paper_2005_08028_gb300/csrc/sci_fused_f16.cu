// Temporally blocked FGP kernels (the implementation is sci_fused.cuh),
// instantiated for __half storage.
#define SCI_FUSED_STORAGE __half
#include "sci_fused.cuh"
