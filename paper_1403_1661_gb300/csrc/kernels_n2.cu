// Kernels for polynomial order 2.
#define SWE_ORDER 2
#include "kernels_order.inc"
