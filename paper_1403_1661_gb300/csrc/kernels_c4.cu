// Kernels for the nodal-collocation variant of polynomial order 4.
#define SWE_ORDER 20
#include "kernels_order.inc"
