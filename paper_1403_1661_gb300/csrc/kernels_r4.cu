// Kernels for the rules of integration order 2N, polynomial order 4.
#define SWE_ORDER 36
#include "kernels_order.inc"
