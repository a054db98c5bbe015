// Kernels for polynomial order 5.
#define SWE_ORDER 5
#include "kernels_order.inc"
