// Kernels for the nodal-collocation variant of polynomial order 2.
#define SWE_ORDER 18
#include "kernels_order.inc"
