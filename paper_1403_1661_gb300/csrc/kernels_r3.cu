// Kernels for the rules of integration order 2N, polynomial order 3.
#define SWE_ORDER 35
#include "kernels_order.inc"
