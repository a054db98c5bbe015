// Kernels for polynomial order 4.
#define SWE_ORDER 4
#include "kernels_order.inc"
