// Final reduction: per-item FP64 partials -> weighted per-triplet energies ->
// E_(T), one CTA per job of the batch.  Both stages use Neumaier's compensated
// summation (Neumaier 1974) in a fixed order, so each job's result is bitwise
// reproducible and independent of the other jobs in the batch.
#include "tc_internal.cuh"

namespace tc {
namespace {

struct Comp { double s, c; };

__device__ __forceinline__ void neumaier_add(Comp &a, double x) {
  const double t = a.s + x;
  a.c += (fabs(a.s) >= fabs(x)) ? ((a.s - t) + x) : ((x - t) + a.s);
  a.s = t;
}

constexpr int RT = 256;

// Thread q handles triplets q, q + RT, ...: each triplet's item partials are
// summed in order and weighted; the thread keeps a compensated sum of its
// triplets; thread 0 combines the RT sums in thread order.
__global__ void __launch_bounds__(RT) reduce_jobs(const __grid_constant__ RedBatch B) {
  const RedJob &J = B.job[blockIdx.x];
  __shared__ double ss[RT], sc[RT], sa[RT], s5[RT], c5[RT];
  Comp a{0.0, 0.0}, a5{0.0, 0.0};
  double absum = 0.0;
  for (int t = threadIdx.x; t < J.n_trip; t += RT) {
    Comp p{0.0, 0.0}, p5{0.0, 0.0};
    const double *pp = J.partial + 2LL * t * J.items_per_trip;
    for (int c = 0; c < J.items_per_trip; ++c) {
      neumaier_add(p, pp[2 * c]);
      neumaier_add(p5, pp[2 * c + 1]);
    }
    const int4 tr = J.trip[t];
    const double e = (double)tr.w * (p.s + p.c);          // weight 1 or 2: exact
    J.e_trip[t] = e;
    if (J.e_ijk) J.e_ijk[((long long)tr.x * J.o + tr.y) * J.o + tr.z] = e;
    neumaier_add(a, e);
    neumaier_add(a5, (double)tr.w * (p5.s + p5.c));
    absum += fabs(e);
  }
  ss[threadIdx.x] = a.s;
  sc[threadIdx.x] = a.c;
  sa[threadIdx.x] = absum;
  s5[threadIdx.x] = a5.s;
  c5[threadIdx.x] = a5.c;
  __syncthreads();
  if (threadIdx.x == 0) {
    Comp tot{0.0, 0.0}, tot5{0.0, 0.0};
    double ab = 0.0, cc = 0.0, cc5 = 0.0;
    for (int i = 0; i < RT; ++i) {
      neumaier_add(tot, ss[i]); cc += sc[i]; ab += sa[i];
      neumaier_add(tot5, s5[i]); cc5 += c5[i];
    }
    J.out[0] = tot.s + (tot.c + cc);
    J.out[1] = ab;
    J.out[2] = tot5.s + (tot5.c + cc5);
  }
}

}  // namespace

cudaError_t launch_reduce(const RedBatch &b, cudaStream_t st) {
  if (b.njobs <= 0) return cudaSuccess;
  reduce_jobs<<<b.njobs, RT, 0, st>>>(b);
  return cudaGetLastError();
}

}  // namespace tc
