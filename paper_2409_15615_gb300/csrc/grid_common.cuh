// Cell indexing shared by the grid build and the grid searches.
#pragma once

#include "kmx_internal.cuh"

// The grid enlarges the requested cell edge by this relative margin; with the
// cell index computed in FP64, two points closer than the requested edge can
// never land in cells two apart, so the 27-cell stencil is always complete.
#define KMX_CELL_MARGIN 1e-6

// floor(x / cell) as floor(x * inv_cell) in FP64; false if it does not fit
// in the 21-bit key field with room for the +-1 stencil offsets.
__device__ __forceinline__ bool kmx_cell_index(float x, double inv_cell, int* c)
{
    double q = floor((double)x * inv_cell);
    if (!(fabs(q) < 1048574.0)) return false;
    *c = (int)q;
    return true;
}
