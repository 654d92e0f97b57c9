// Temporally blocked FGP kernels (the implementation is sci_fused.cuh),
// instantiated for __nv_bfloat16 storage.
#define SCI_FUSED_STORAGE __nv_bfloat16
#include "sci_fused.cuh"
