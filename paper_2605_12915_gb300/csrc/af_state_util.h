// af_state_util.h -- host-side helpers on the FP64 state descriptor of the C ABI
// (af_state_f64, include/af.h), shared by the handle API and the
// allocation-free step.
#pragma once

#include <stddef.h>

#include "../../include/af.h"

namespace af {

// Plane p of a state in the ABI's order: averages 0-3, vertex 4-7, x-edge
// midpoints 8-11, y-edge midpoints 12-15.
inline const double* state_plane(const af_state_f64* s, int p) {
  if (p < 4) return s->avg[p];
  if (p < 8) return s->vtx[p - 4];
  if (p < 12) return s->ev[p - 8];
  return s->eh[p - 12];
}

// true when some plane of a and some plane of b (each `bytes` long) share a byte
inline bool state_planes_overlap(const af_state_f64* a, const af_state_f64* b, size_t bytes) {
  for (int p = 0; p < 16; ++p)
    for (int q = 0; q < 16; ++q) {
      const char* x = (const char*)state_plane(a, p);
      const char* y = (const char*)state_plane(b, q);
      if (x < y + bytes && y < x + bytes) return true;
    }
  return false;
}

}  // namespace af
