// Domain decomposition of a hexahedral mesh (host side): a recursive coordinate bisection of the
// element centroids, and the extraction of one part with the lists of interfaces it shares with
// other parts (the halo).
//
// The paper distributes the mesh over MPI ranks and pairs the faces on partition boundaries
// (section "Pre-processing", Algorithm 2, "MatchMPIFaces"); each time step then exchanges the
// data of those faces.  Here every part is built from the global connectivity of the whole mesh,
// so both sides of a shared interface carry the same interface record (side numbering and
// orientation code of the global mesh): the trace a part writes into its own slot is directly
// the trace its neighbour needs in the other slot of the same interface.  Shared interfaces are
// listed per peer part in ascending global interface number, on both sides, so the k-th entry a
// part sends to a peer is the k-th entry that peer receives from it.
#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "fr_part.hpp"

namespace frx {

namespace {

// Splits idx[lo, hi) (element indices) into `parts` groups of near-equal weight by recursive
// bisection along the longest extent of their centroids; part ids start at `first`.
void rcb(std::vector<int64_t> &idx, int64_t lo, int64_t hi, const std::vector<double> &cent,
         const std::vector<double> &w, int parts, int first, std::vector<int32_t> &part) {
  if (parts <= 1 || hi - lo <= 1) {
    for (int64_t i = lo; i < hi; ++i) part[idx[i]] = first;
    return;
  }
  double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = lo; i < hi; ++i)
    for (int c = 0; c < 3; ++c) {
      mn[c] = std::min(mn[c], cent[idx[i] * 3 + c]);
      mx[c] = std::max(mx[c], cent[idx[i] * 3 + c]);
    }
  int ax = 0;
  for (int c = 1; c < 3; ++c)
    if (mx[c] - mn[c] > mx[ax] - mn[ax]) ax = c;
  // Stable order along the axis (ties by element index) so the split is deterministic.
  std::stable_sort(idx.begin() + lo, idx.begin() + hi, [&](int64_t a, int64_t b) {
    const double xa = cent[a * 3 + ax], xb = cent[b * 3 + ax];
    return xa < xb || (xa == xb && a < b);
  });
  const int left = parts / 2;
  double total = 0.0;
  for (int64_t i = lo; i < hi; ++i) total += w[idx[i]];
  const double target = total * left / parts;
  double acc = 0.0;
  int64_t cut = lo;
  while (cut < hi - 1 && acc + 0.5 * w[idx[cut]] < target) acc += w[idx[cut++]];
  cut = std::max(cut, lo + 1);
  rcb(idx, lo, cut, cent, w, left, first, part);
  rcb(idx, cut, hi, cent, w, parts - left, first + left, part);
}

}  // namespace

fr_status partition_elements(const std::vector<double> &cent, const std::vector<double> &w, int n_parts,
                             std::vector<int32_t> &part, std::string &err) {
  const int64_t n = (int64_t)w.size();
  if (n_parts < 1) {
    err = "n_parts must be at least 1";
    return FR_EINVAL;
  }
  if (n_parts > n) {
    err = "more parts than elements";
    return FR_EINVAL;
  }
  std::vector<int64_t> idx((size_t)n);
  std::iota(idx.begin(), idx.end(), 0);
  part.assign((size_t)n, 0);
  rcb(idx, 0, n, cent, w, n_parts, 0, part);
  return FR_OK;
}

fr_status extract_part(const HostMesh &g, const std::vector<int32_t> &part, int rank, HostMesh &m, HaloLists &halo,
                       std::string &err) {
  const int64_t G = g.E + g.Ep;   // global elements: hexahedra, then prisms
  if ((int64_t)part.size() != G) {
    err = "partition has the wrong length";
    return FR_EINVAL;
  }
  const int Np = g.Np, Nf = g.Nf, Npp = g.Npp;
  // Local numbering keeps the global layout: the part's hexahedra, then its prisms.
  std::vector<int64_t> g2l((size_t)G, -1);
  halo = HaloLists{};
  int64_t E = 0, Ep = 0;
  for (int64_t e = 0; e < g.E; ++e)
    if (part[e] == rank) {
      g2l[e] = E++;
      halo.elem_global.push_back(e);
    }
  for (int64_t e = g.E; e < G; ++e)
    if (part[e] == rank) {
      g2l[e] = E + Ep++;
      halo.elem_global.push_back(e);
    }
  if (E + Ep == 0) {
    err = "the part owns no element";
    return FR_EINVAL;
  }
  // Local interfaces: two-sided ones with at least one owned side (global order), then the
  // boundary faces of owned elements.
  std::vector<int64_t> l2g_if;
  std::vector<int64_t> gif2l((size_t)g.n_if, -1);
  struct Shared {
    int32_t peer;
    int64_t gid, iface;
    int8_t side;
  };
  std::vector<Shared> shared;
  for (int64_t I = 0; I < g.n_interior; ++I) {
    const int32_t eL = g.if_elem[2 * I], eR = g.if_elem[2 * I + 1];
    const bool oL = g2l[eL] >= 0, oR = g2l[eR] >= 0;
    if (!oL && !oR) continue;
    gif2l[I] = (int64_t)l2g_if.size();
    if (oL != oR) shared.push_back({part[oL ? eR : eL], I, gif2l[I], (int8_t)(oL ? 0 : 1)});
    l2g_if.push_back(I);
  }
  const int64_t n_interior = (int64_t)l2g_if.size();
  for (int64_t I = g.n_interior; I < g.n_if; ++I)
    if (g2l[g.if_elem[2 * I]] >= 0) {
      gif2l[I] = (int64_t)l2g_if.size();
      l2g_if.push_back(I);
    }
  const int64_t n_if = (int64_t)l2g_if.size();
  if (n_if >= (int64_t(1) << 27)) {
    err = "too many interfaces for the packed face table";
    return FR_EINVAL;
  }

  m = HostMesh{};
  m.p = g.p;
  m.N = g.N;
  m.Np = Np;
  m.Nf = Nf;
  m.E = E;
  m.n_if = n_if;
  m.n_interior = n_interior;
  m.bcs = g.bcs;
  m.ef.resize((size_t)E * 6);
  m.metrics.resize((size_t)E * 10 * Np);
  m.liftfac.resize((size_t)E * 6 * 3 * Nf);
  m.xsol.resize(((size_t)E * Np + (size_t)Ep * Npp) * 3);
  m.h.resize((size_t)(E + Ep));
  auto remap = [&](int32_t packed) { return (int32_t)((gif2l[packed >> 4] << 4) | (packed & 15)); };
  for (int64_t le = 0; le < E; ++le) {
    const int64_t e = halo.elem_global[le];
    for (int f = 0; f < 6; ++f) m.ef[le * 6 + f] = remap(g.ef[e * 6 + f]);
    std::copy_n(g.metrics.begin() + e * 10 * Np, 10 * Np, m.metrics.begin() + le * 10 * Np);
    std::copy_n(g.liftfac.begin() + e * 18 * Nf, 18 * Nf, m.liftfac.begin() + le * 18 * Nf);
    std::copy_n(g.xsol.begin() + e * Np * 3, Np * 3, m.xsol.begin() + le * Np * 3);
    m.h[le] = g.h[e];
  }
  if (g.Ep > 0) {
    m.Ep = Ep;
    m.Nt = g.Nt;
    m.Npp = Npp;
    m.ptab = g.ptab;
    m.tri_slot = g.tri_slot;
    m.ef_p.resize((size_t)Ep * 5);
    m.metrics_p.resize((size_t)Ep * 10 * Npp);
    for (int64_t lp = 0; lp < Ep; ++lp) {
      const int64_t e = halo.elem_global[E + lp], ep = e - g.E;
      for (int f = 0; f < 5; ++f) m.ef_p[lp * 5 + f] = remap(g.ef_p[ep * 5 + f]);
      std::copy_n(g.metrics_p.begin() + ep * 10 * Npp, 10 * Npp, m.metrics_p.begin() + lp * 10 * Npp);
      std::copy_n(g.xsol.begin() + (g.E * Np + ep * Npp) * 3, Npp * 3, m.xsol.begin() + (E * Np + lp * Npp) * 3);
      m.h[E + lp] = g.h[e];
    }
    m.if_tri.resize((size_t)n_if);
    for (int64_t li = 0; li < n_if; ++li) m.if_tri[li] = g.if_tri[l2g_if[li]];
  }
  m.if_bc.resize((size_t)n_if);
  m.if_elem.resize((size_t)n_if * 2);
  m.if_up.resize((size_t)n_if);
  m.normals.resize((size_t)n_if * 4 * Nf);
  for (int64_t li = 0; li < n_if; ++li) {
    const int64_t I = l2g_if[li];
    m.if_bc[li] = g.if_bc[I];
    for (int s = 0; s < 2; ++s) {
      const int32_t e = g.if_elem[2 * I + s];
      m.if_elem[2 * li + s] = (e >= 0 && g2l[e] >= 0) ? (int32_t)g2l[e] : -1;
    }
    m.if_up[li] = g.if_up[I];
    std::copy_n(g.normals.begin() + I * 4 * Nf, 4 * Nf, m.normals.begin() + li * 4 * Nf);
  }
  // Halo lists, per peer in ascending global interface number.
  std::sort(shared.begin(), shared.end(), [](const Shared &a, const Shared &b) {
    return a.peer < b.peer || (a.peer == b.peer && a.gid < b.gid);
  });
  for (const Shared &s : shared) {
    if (halo.peers.empty() || halo.peers.back() != s.peer) {
      halo.peers.push_back(s.peer);
      halo.peer_begin.push_back((int64_t)halo.iface.size());
    }
    halo.iface.push_back(s.iface);
    halo.side.push_back(s.side);
    halo.gid.push_back(s.gid);
  }
  halo.peer_begin.push_back((int64_t)halo.iface.size());
  return FR_OK;
}

}  // namespace frx
