// Triple-double (L = 3) instantiation of the C entry points.
#include "lu_host.cuh"
MCLU_DEFINE_PRECISION(td, 3)
