// Kernels for the nodal-collocation variant of polynomial order 3.
#define SWE_ORDER 19
#include "kernels_order.inc"
