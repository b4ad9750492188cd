// Stencil kernels: f32 transport, WENO3_C4 scheme.
#define APD_T float
#define APD_SCHEME WENO3_C4
#define APD_NAME stencil_f32_w3
#include "stencil_tu.inc"
