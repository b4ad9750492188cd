// Stencil kernels: f64 transport, WENO5_C4 scheme.
#define APD_T double
#define APD_SCHEME WENO5_C4
#define APD_NAME stencil_f64_w5
#include "stencil_tu.inc"
