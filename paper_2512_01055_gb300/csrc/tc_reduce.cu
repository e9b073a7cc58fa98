// Final reduction: per-item FP64 partials -> weighted per-triplet energies ->
// E_(T).  Both stages use Neumaier's compensated summation (Neumaier 1974) in
// a fixed order, so the result is bitwise reproducible.
#include "tc_internal.cuh"

namespace tc {
namespace {

struct Comp { double s, c; };

__device__ __forceinline__ void neumaier_add(Comp &a, double x) {
  const double t = a.s + x;
  a.c += (fabs(a.s) >= fabs(x)) ? ((a.s - t) + x) : ((x - t) + a.s);
  a.s = t;
}

// One thread per triplet: e_trip[t] = weight * sum of the triplet's item partials.
__global__ void reduce_triplets(Dims d, Work w, double *e_trip, double *e_ijk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= d.n_trip) return;
  Comp a{0.0, 0.0};
  const double *p = w.partial + (long long)t * d.items_per_trip;
  for (int c = 0; c < d.items_per_trip; ++c) neumaier_add(a, p[c]);
  const int4 tr = w.trip[t];
  const double e = (double)tr.w * (a.s + a.c);      // weight 1 or 2: exact
  e_trip[t] = e;
  if (e_ijk) e_ijk[((long long)tr.x * d.o + tr.y) * d.o + tr.z] = e;
}

// One block: E = compensated sum of e_trip[0 .. n); out[0] = E, out[1] = sum |e|.
constexpr int RT = 256;
__global__ void reduce_total(const double *e_trip, int n, double *out) {
  __shared__ double ss[RT], sc[RT], sa[RT];
  Comp a{0.0, 0.0};
  double absum = 0.0;
  for (int i = threadIdx.x; i < n; i += RT) { neumaier_add(a, e_trip[i]); absum += fabs(e_trip[i]); }
  ss[threadIdx.x] = a.s; sc[threadIdx.x] = a.c; sa[threadIdx.x] = absum;
  __syncthreads();
  if (threadIdx.x == 0) {
    Comp tot{0.0, 0.0};
    double ab = 0.0, cc = 0.0;
    for (int i = 0; i < RT; ++i) { neumaier_add(tot, ss[i]); cc += sc[i]; ab += sa[i]; }
    out[0] = tot.s + (tot.c + cc);
    out[1] = ab;
  }
}

}  // namespace

cudaError_t launch_reduce(const Dims &d, const Work &w, double *e_trip, double *e_ijk, double *out,
                          cudaStream_t st) {
  if (d.n_trip > 0) {
    reduce_triplets<<<(d.n_trip + 255) / 256, 256, 0, st>>>(d, w, e_trip, e_ijk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  reduce_total<<<1, RT, 0, st>>>(e_trip, d.n_trip, out);
  return cudaGetLastError();
}

}  // namespace tc
