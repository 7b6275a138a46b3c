// Double-double (L = 2) instantiation of the C entry points.
#include "lu_host.cuh"
MCLU_DEFINE_PRECISION(dd, 2)
