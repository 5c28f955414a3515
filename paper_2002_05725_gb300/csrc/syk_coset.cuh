// Member sets of the X-mask cosets the coset matvecs run as unrolled bodies (syk_terms.cpp,
// coset_layout_host, lists the same sets in the same order).
//
// Row-slot offset d (bit d of a set) is the value of a mask's RB row-slot bits.  Compact
// masks have popcount 4, or 3 when the top spin is one of the four (its bit is dropped with
// the parity sector), so the masks of one coset share the bits outside the row-slot bits
// and have popcount 3 - w or 4 - w inside, w the popcount outside.
#pragma once

#include <cstdint>

namespace syk {

template <int RB>
struct CosetShapes;
template <>
struct CosetShapes<1> {
  static constexpr uint32_t n = 1, s0 = 0x3u, s1 = 0u, s2 = 0u;
};
template <>
struct CosetShapes<2> {
  static constexpr uint32_t n = 2, s0 = 0x7u, s1 = 0xEu, s2 = 0u;
};
template <>
struct CosetShapes<3> {
  static constexpr uint32_t n = 3, s0 = 0x17u, s1 = 0xE8u, s2 = 0x7Eu;
};

}  // namespace syk
