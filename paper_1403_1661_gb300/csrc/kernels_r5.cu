// Kernels for the rules of integration order 2N, polynomial order 5.
#define SWE_ORDER 37
#include "kernels_order.inc"
