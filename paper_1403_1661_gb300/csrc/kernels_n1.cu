// Kernels for polynomial order 1.
#define SWE_ORDER 1
#include "kernels_order.inc"
