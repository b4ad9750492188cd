// Stencil kernels: f64 transport, WENO3_C4 scheme.
#define APD_T double
#define APD_SCHEME WENO3_C4
#define APD_NAME stencil_f64_w3
#include "stencil_tu.inc"
