// Instantiations of the single-frame and the persistent many-frame reconstruction kernels for
// polynomial order M = 1.
#include "lpa_orders.cuh"

LPA_ORDER_ENTRY_POINTS(1)
