// The second level of a cloud's bounding-sphere index.
//
// The first level is one sphere per kSphereTile consecutive points of the
// Morton-ordered prepass array (Cloud::spheres[0 .. n_spheres)).  Every
// kGroupSpheres consecutive spheres also have a group sphere, stored after
// the spheres in the same allocation (Cloud::spheres[n_spheres + g]).  A group
// sphere (centre C_g, radius R_g) contains each member sphere whole:
// R_g >= |c_t - C_g| + r_t, so |x - C_g| - R_g is a lower bound on both
// |x - c_t| - r_t and |x - c_t| + r_t for every member t, and a search skips a
// group when that bound rules out all of its members at once.
#pragma once

#include <cstdint>

namespace ptsdf {

constexpr int kGroupSpheres = 64;   // spheres per group sphere

inline int64_t group_count(int64_t n_spheres) { return (n_spheres + kGroupSpheres - 1) / kGroupSpheres; }

}  // namespace ptsdf
