// Domain decomposition (host side): partition of the elements and extraction of one part with its
// halo lists.  See fr_part.cpp.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fr_internal.hpp"

namespace frx {

// Interfaces a part shares with other parts, grouped by peer (ascending rank), each group in
// ascending global interface number.  Entry k: local interface iface[k], this part's side
// side[k] (the peer writes the other slot), global interface gid[k].
struct HaloLists {
  std::vector<int32_t> peers;
  std::vector<int64_t> peer_begin;     // [n_peers + 1]
  std::vector<int64_t> iface, gid;
  std::vector<int8_t> side;
  std::vector<int64_t> elem_global;    // [E] global element of each local element
};

// Recursive coordinate bisection of element centroids cent [n][3] into n_parts parts of near-equal
// total weight w [n] (the work of an element, e.g. its solution points); part[e] in [0, n_parts).
// Each cut is across the longest extent of the group's centroids; ties are ordered by index, so
// the result is deterministic.
fr_status partition_elements(const std::vector<double> &cent, const std::vector<double> &w, int n_parts,
                             std::vector<int32_t> &part, std::string &err);

// The part `rank` of the global mesh g: its elements (global order), the interfaces touching
// them (two-sided first, then boundary faces) with the global records, and its halo lists.
fr_status extract_part(const HostMesh &g, const std::vector<int32_t> &part, int rank, HostMesh &local,
                       HaloLists &halo, std::string &err);

}  // namespace frx
