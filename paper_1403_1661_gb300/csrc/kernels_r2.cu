// Kernels for the rules of integration order 2N, polynomial order 2.
#define SWE_ORDER 34
#include "kernels_order.inc"
