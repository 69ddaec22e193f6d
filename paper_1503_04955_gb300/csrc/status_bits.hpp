// Bits of a plan's device status word.
#pragma once
#include <cstdint>

namespace dkss {
enum : uint32_t {
    kStatusCarryOut = 1u,  // the product overflowed 2N bits (inconsistent coefficients)
    kStatusTimeout = 2u,   // a bounded device-side wait gave up
    kStatusRange = 4u      // DKSS_DEBUG_CHECKS: a residue at a stage boundary was not below p^z
};
}  // namespace dkss
