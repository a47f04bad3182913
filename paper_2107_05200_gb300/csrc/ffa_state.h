// Host-only conversion between the per-element state of Algorithm 1 (U, P,
// Lambda as d x d matrices) and the layout the library keeps on the device.
#pragma once

#include <cstdint>
#include <string>

namespace ffa {

// Device layout, structure of arrays (component k of element i at k*m + i):
// U as (cos, sin) in 2D or the unit quaternion (w, x, y, z) in 3D, P as its
// upper triangle row by row (p00 p01 p11 / p00 p01 p02 p11 p12 p22), Lambda as
// its d*d entries (row a, column k at (a*d + k)*m + i).
constexpr int state_u_size(int d) { return d == 2 ? 2 : 4; }
constexpr int state_p_size(int d) { return d == 2 ? 3 : 6; }

// Device layout (as doubles) -> d x d matrices, row-major, element after element.
void unpack_state(int d, int64_t m, const double* u, const double* p, const double* l, double* U, double* P,
                  double* Lam);

// d x d matrices -> device layout (as doubles).  U must be a rotation to 1e-5
// (|U^T U - I| and |det U - 1|, entrywise); P is symmetrized.  Returns false,
// with msg naming the element, on a non-rotation U or a non-finite entry.
bool pack_state(int d, int64_t m, const double* U, const double* P, const double* Lam, double* u, double* p, double* l,
                std::string& msg);

}  // namespace ffa
