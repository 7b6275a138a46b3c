// Quadruple-double (L = 4) instantiation of the C entry points.
#include "lu_host.cuh"
MCLU_DEFINE_PRECISION(qd, 4)
