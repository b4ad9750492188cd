// Stencil kernels: f32 transport, WENO5_C4 scheme.
#define APD_T float
#define APD_SCHEME WENO5_C4
#define APD_NAME stencil_f32_w5
#include "stencil_tu.inc"
