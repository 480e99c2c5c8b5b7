// rest_host.h -- host view of the compensated FP32 rest population (lbmk::rest_update): the
// rest population of a cell is hi + q u, hi the FP32 value of plane 0, q the int16 of the
// buffer's tenth plane and u = 2^(e - 38) the lattice's unit, e the binary exponent of the
// Carnahan-Starling packing limit 4/b.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

namespace lbm_host {

// The unit u of a lattice with EOS co-volume b, and its inverse.
inline double rest_unit(double b) { return std::ldexp(1.0, std::ilogb(4.0 / b) - 38); }
inline double rest_inv(double b) { return std::ldexp(1.0, 38 - std::ilogb(4.0 / b)); }

// The FP64 value of (hi, q).
inline double rest_decode(float hi, short q, double unit) { return (double)hi + (double)q * unit; }

// q of an FP64 value v whose FP32 rounding is hi.
inline short rest_encode(double v, float hi, double inv) {
    const double q = std::nearbyint((v - (double)hi) * inv);
    return (short)std::max(-32767.0, std::min(32767.0, q));
}

}  // namespace lbm_host
