// Internal declarations shared by the CUDA sources of the (T) library.
//
// Work decomposition (both precisions):
//   * occupied triplets i >= j >= k, all-equal triplets dropped (their sum is
//     exactly zero, Eq. 1), each with weight 2 - d_ij - d_jk;
//   * the virtual range [0, v) cut into tiles of edge NT; an "orbit" is a tile
//     triple P >= Q >= R.  The points (a, b, c) with a in P, b in Q, c in R and
//     a >= b >= c are the canonical points; W at the six permutations of each
//     canonical point lies in the six permuted tile blocks (P,Q,R), (P,R,Q),
//     (Q,P,R), (Q,R,P), (R,P,Q), (R,Q,P) of the same orbit, so one orbit holds
//     everything the energy bracket of Eq. 1 needs;
//   * a work item is (triplet, chunk of consecutive orbits); each item writes
//     one FP64 partial, so the result does not depend on which CTA ran it.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

struct Dims {
  int o, v;
  int nt;              // tile edge
  int ntiles;          // ceil(v / nt)
  int n_trip;          // triplets i >= j >= k without i == j == k
  int n_orb;           // tile triples P >= Q >= R
  int orb_per_item;
  int items_per_trip;
  long long n_items;
};

struct Inputs {        // device pointers, layouts as in include/tc.h
  const double *eps, *t1, *t2, *ovvv, *ovoo, *ovov;
};

struct Work {
  const int4 *trip;    // (i, j, k, weight)
  const int4 *orb;     // (P, Q, R, 0) tile indices
  double *partial;     // [n_items]
  unsigned int *counter;
  int *err;            // device error flag (0 = fine)
};

// The six permutations of three positions, in the order
// (abc), (acb), (bac), (bca), (cab), (cba); entries 0, 3, 4 are even.
__host__ __device__ constexpr int perm3(int s, int pos) {
  return (s == 0) ? pos
       : (s == 1) ? (pos == 0 ? 0 : (pos == 1 ? 2 : 1))
       : (s == 2) ? (pos == 0 ? 1 : (pos == 1 ? 0 : 2))
       : (s == 3) ? (pos == 0 ? 1 : (pos == 1 ? 2 : 0))
       : (s == 4) ? (pos == 0 ? 2 : (pos == 1 ? 0 : 1))
       :            (pos == 0 ? 2 : (pos == 1 ? 1 : 0));
}
__host__ __device__ constexpr bool perm3_even(int s) { return s == 0 || s == 3 || s == 4; }

// Host-side launchers (defined in the .cu files).
cudaError_t launch_fp64(const Dims &d, const Inputs &in, const Work &w, int grid, cudaStream_t st);
int fp64_tile();
size_t fp64_smem_bytes();
cudaError_t fp64_blocks_per_sm(int *n);
cudaError_t launch_reduce(const Dims &d, const Work &w, double *e_trip, double *e_ijk, double *out,
                          cudaStream_t st);

// Split-precision path (tc_split.cu): byte offsets of the BF16 slices and FP32
// copies inside its workspace.
struct SplitLayout {
  int vpad, opad;                          // row pitches (elements), multiples of 8
  size_t ovvv, t2, t2h, ovoo, t1f, ovovf;  // offsets
  size_t total;
};
int split_tile();
SplitLayout split_layout(int o, int v, int S);
cudaError_t launch_split_prep(const Dims &d, int S, const Inputs &in, void *ws, const SplitLayout &L, cudaStream_t st);
cudaError_t launch_split(const Dims &d, int S, const Inputs &in, void *ws, const SplitLayout &L, const Work &w,
                         int num_sms, cudaStream_t st);

}  // namespace tc
