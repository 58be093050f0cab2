// Host-side facet connectivity of a conforming affine simplicial mesh
// (Sec. 2, "Preliminaries": every facet belongs to one or two elements).
//
// Each element's vertex ids are sorted, local facet f is the facet opposite
// the f-th vertex, and facets are numbered by sorting their vertex tuples
// lexicographically.  The lower-index element of a facet owns it (its
// outward normal orients the facet's H(div) moments).
#include <algorithm>
#include <array>
#include <string>

#include "dgc_internal.h"

namespace dgc {

std::string build_connectivity(int D, int n_vert, int n_elem, std::vector<int>& elems, Connectivity& out) {
  const int NF = D + 1;
  for (int e = 0; e < n_elem; ++e) {
    int* v = &elems[(size_t)e * NF];
    for (int a = 0; a < NF; ++a)
      if (v[a] < 0 || v[a] >= n_vert)
        return "element " + std::to_string(e) + " references vertex " + std::to_string(v[a]) + " out of range";
    std::sort(v, v + NF);
    for (int a = 1; a < NF; ++a)
      if (v[a] == v[a - 1]) return "element " + std::to_string(e) + " repeats a vertex";
  }
  struct FK {
    std::array<int, 3> v;
    int e, f;
  };
  std::vector<FK> keys((size_t)n_elem * NF);
  for (int e = 0; e < n_elem; ++e)
    for (int f = 0; f < NF; ++f) {
      FK& kk = keys[(size_t)e * NF + f];
      kk.v = {-1, -1, -1};
      int n = 0;
      for (int a = 0; a < NF; ++a)
        if (a != f) kk.v[n++] = elems[(size_t)e * NF + a];
      kk.e = e;
      kk.f = f;
    }
  std::sort(keys.begin(), keys.end(), [](const FK& a, const FK& b) {
    if (a.v != b.v) return a.v < b.v;
    return a.e < b.e;
  });
  out.nbr.assign((size_t)n_elem * NF, -1);
  out.facet_id.assign((size_t)n_elem * NF, -1);
  out.orient.assign((size_t)n_elem * NF, 1);
  out.sides.clear();
  int nF = 0;
  for (size_t j = 0; j < keys.size();) {
    size_t l = j + 1;
    while (l < keys.size() && keys[l].v == keys[j].v) ++l;
    if (l - j > 2) return "a facet is shared by " + std::to_string(l - j) + " elements: mesh is not conforming";
    const FK& a = keys[j];
    out.facet_id[(size_t)a.e * NF + a.f] = nF;
    out.sides.push_back((a.e << 2) | a.f);
    if (l - j == 2) {
      const FK& b = keys[j + 1];
      out.facet_id[(size_t)b.e * NF + b.f] = nF;
      out.nbr[(size_t)a.e * NF + a.f] = (b.e << 2) | b.f;
      out.nbr[(size_t)b.e * NF + b.f] = (a.e << 2) | a.f;
      out.orient[(size_t)b.e * NF + b.f] = -1;
      out.sides.push_back((b.e << 2) | b.f);
    } else {
      out.sides.push_back(-1);
    }
    ++nF;
    j = l;
  }
  out.n_facets = nF;
  return std::string();
}

}  // namespace dgc
