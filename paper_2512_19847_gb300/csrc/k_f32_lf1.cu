// Stencil kernels: f32 transport, LF1_C2 scheme.
#define APD_T float
#define APD_SCHEME LF1_C2
#define APD_NAME stencil_f32_lf1
#include "stencil_tu.inc"
