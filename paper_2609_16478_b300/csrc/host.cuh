// Host-side helpers shared between translation units (internal).
#pragma once

#include "ahoc.h"
#include "common.cuh"

namespace ahoc {
// grid geometry from the public arguments (argument checks included)
ahoc_status host_make_geom(int dim, const int64_t* N, const double* lo, const double* hi, Geom* g);
// stencil coefficients of the plan's grid
Coefs host_make_coefs(const Geom& g);
// record the thread's last error message and return s
ahoc_status host_fail(ahoc_status s, const char* msg);
// which tridiagonal form a grid uses, and its chunk length
bool host_tri_chunked(const Geom& g);
int host_tri_chunk_len(const Geom& g);
}  // namespace ahoc
