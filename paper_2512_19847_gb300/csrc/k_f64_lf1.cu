// Stencil kernels: f64 transport, LF1_C2 scheme.
#define APD_T double
#define APD_SCHEME LF1_C2
#define APD_NAME stencil_f64_lf1
#include "stencil_tu.inc"
