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
//
// Every kernel takes a batch of up to MAX_BATCH independent jobs by value;
// the global item range is the concatenation of the jobs' item ranges.  A
// job's result depends only on its own items, so it is the same alone or in
// any batch.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tc {

constexpr int MAX_BATCH = 32;

struct Dims {
  int o, v;
  int nt;              // tile edge
  int ntiles;          // ceil(v / nt)
  int n_trip;          // triplets processed (all i >= j >= k without i == j == k, or a subset)
  int n_orb;           // tile triples P >= Q >= R
  int orb_per_item;
  int items_per_trip;
  long long n_items;
};

// Work item q of a job (its sequence number in launch order) -> (triplet t,
// orbit chunk c).  Items run chunk-major: the CTAs in flight at one time work
// on the same few tile triples for many triplets, so the operand tiles they
// stream are shared through L2.  The item's partial keeps the triplet-major
// slot t * items_per_trip + c, so the order of the final reduction (and every
// bit of the result) does not depend on the launch order.
__host__ __device__ inline long long item_slot(const Dims &d, long long q, int &t, int &chunk) {
  chunk = (int)(q / d.n_trip);
  t = (int)(q % d.n_trip);
  return (long long)t * d.items_per_trip + chunk;
}

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

// ---------------------------------------------------------------- FP64 path
struct FpJob {
  Dims d;
  Inputs in;
  Work w;
  long long item0;     // first global item of this job in the launch
  long long item_base; // the job's own index of that item (a launch may run a slice of a job)
};
struct FpBatch {
  int njobs;
  long long total_items;
  unsigned int *counter;   // global work counter of the launch (zeroed before it)
  FpJob job[MAX_BATCH];
};
int fp64_tile();
size_t fp64_smem_bytes();
cudaError_t fp64_blocks_per_sm(int *n);
cudaError_t launch_fp64(const FpBatch &b, int grid, cudaStream_t st);
// Kernel-node parameters of one FP64 launch (for CUDA graphs); args[0] must
// point to b while the parameters are used.
void fp64_node_params(const FpBatch &b, int grid, void **args, cudaKernelNodeParams *p);

// ---------------------------------------------------------------- split path
// Byte offsets of the BF16 operand images and FP32 copies inside a job's
// split workspace.
struct SplitLayout {
  int vpad, opad;
  size_t ovvv, t2, t2h, ovoo, t1f, ovovf;
  size_t total;
};
struct SplitJob {
  Dims d;
  int kch_p, kch_h;      // K blocks (of 16) of particle / hole products
  int T;                 // virtual tiles
  const unsigned char *imgA_p, *imgA_h, *imgB_p, *imgB_h;   // operand images
  const float *t1f, *ovovf;
  const double *eps;
  Work w;
  long long item0;       // first global item of this job in the launch
  long long item_base;   // the job's own index of that item
  long long n_run;       // items of this job in the launch (0: all n_items)
};
struct SplitBatch {
  int njobs;
  int stages;            // set by launch_split
  long long total_items;
  int *err;
  SplitJob job[MAX_BATCH];
};
int split_tile();
SplitLayout split_layout(int o, int v, int S);
cudaError_t launch_split_prep(const Dims &d, int S, const Inputs &in, void *ws, const SplitLayout &L, cudaStream_t st);
SplitJob split_job(const Dims &d, const Inputs &in, const void *ws, const SplitLayout &L, const Work &w);
cudaError_t launch_split(SplitBatch &b, int S, int num_sms, cudaStream_t st);
// Prepare b (item offsets, stages) and fill kernel-node parameters of the launch
// launch_split would make; also performs launch_split's one-time set-up.
cudaError_t split_node_params(SplitBatch &b, int S, int grid, void **args, cudaKernelNodeParams *p, cudaStream_t st);

// ---------------------------------------------------------------- reduction
struct RedJob {
  int n_trip, items_per_trip, o;
  const int4 *trip;
  const double *partial;
  double *e_trip;        // [n_trip] weighted triplet contributions
  double *e_ijk;         // optional [o][o][o]
  double *out;           // [2]: E and sum |e|
};
struct RedBatch {
  int njobs;
  RedJob job[MAX_BATCH];
};
cudaError_t launch_reduce(const RedBatch &b, cudaStream_t st);

}  // namespace tc
