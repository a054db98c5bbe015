// Kernels for polynomial order 3.
#define SWE_ORDER 3
#include "kernels_order.inc"
