// Kernels for the nodal-collocation variant of polynomial order 5.
#define SWE_ORDER 21
#include "kernels_order.inc"
