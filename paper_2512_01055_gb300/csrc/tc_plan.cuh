// Host-side planning shared by the blocking entry points and the serving
// engine: work decomposition of a job, layout of its workspace, and the
// triplet / orbit tables the kernels read.
#pragma once
#include <algorithm>
#include <vector>

#include "tc_internal.cuh"

namespace tc {
namespace plan {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// n_trip_override >= 0: the job processes that many listed triplets.
// min_opi: fewest orbits per work item.
inline Dims make_dims(int o, int v, int nt, int n_trip_override = -1, int min_opi = 1) {
  Dims d{};
  d.o = o;
  d.v = v;
  d.nt = nt;
  d.ntiles = (v + nt - 1) / nt;
  const long long T = d.ntiles;
  d.n_trip = n_trip_override >= 0 ? n_trip_override : (int)((long long)o * (o + 1) * (o + 2) / 6 - o);
  d.n_orb = (int)(T * (T + 1) * (T + 2) / 6);
  const long long pairs = (long long)d.n_trip * d.n_orb;
  const long long target = 4LL << 20;   // at most ~4M partials
  d.orb_per_item = (int)std::max<long long>(std::max(1, min_opi), (pairs + target - 1) / target);
  d.orb_per_item = std::min(d.orb_per_item, std::max(1, d.n_orb));
  d.items_per_trip = (d.n_orb + d.orb_per_item - 1) / d.orb_per_item;
  d.n_items = (long long)d.n_trip * d.items_per_trip;
  return d;
}

struct Layout {            // byte offsets inside a job's workspace
  size_t trip, orb, partial, e_trip, out, counter, total;
};

inline Layout make_layout(const Dims &d) {
  Layout L{};
  size_t off = 0;
  L.trip = off;    off = align256(off + sizeof(int4) * (size_t)std::max(1, d.n_trip));
  L.orb = off;     off = align256(off + sizeof(int4) * (size_t)std::max(1, d.n_orb));
  L.partial = off; off = align256(off + 2 * sizeof(double) * (size_t)std::max<long long>(1, d.n_items));
  L.e_trip = off;  off = align256(off + sizeof(double) * (size_t)std::max(1, d.n_trip));
  L.out = off;     off = align256(off + 4 * sizeof(double));
  L.counter = off; off = align256(off + 2 * sizeof(unsigned));
  L.total = off;
  return L;
}

// Host image of the triplet table followed (at L.orb - L.trip) by the orbit
// table.  subset: the triplets to process instead of all of them.
inline std::vector<int4> tables(const Dims &d, const Layout &L, const std::vector<int4> *subset) {
  std::vector<int4> h((L.partial - L.trip) / sizeof(int4), make_int4(0, 0, 0, 0));
  int n = 0;
  if (subset) {
    for (const int4 &t : *subset) h[n++] = t;
  } else {
    for (int i = 0; i < d.o; ++i)
      for (int j = 0; j <= i; ++j)
        for (int k = 0; k <= j; ++k) {
          if (i == k) continue;                       // i == j == k: zero contribution
          h[n++] = make_int4(i, j, k, 2 - (i == j) - (j == k));
        }
  }
  int4 *ho = h.data() + (L.orb - L.trip) / sizeof(int4);
  int m = 0;
  for (int P = 0; P < d.ntiles; ++P)
    for (int Q = 0; Q <= P; ++Q)
      for (int R = 0; R <= Q; ++R) ho[m++] = make_int4(P, Q, R, 0);
  return h;
}

// Input bytes of a job held on the device (eps, t1, t2, ovvv, ovoo, ovov).
inline size_t input_bytes(int o, int v) {
  const size_t O = o, V = v;
  return sizeof(double) * (O + V + O * V + O * O * V * V + O * V * V * V + O * V * O * O + O * V * O * V);
}

}  // namespace plan
}  // namespace tc
