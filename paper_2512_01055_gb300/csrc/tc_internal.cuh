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
#include <cuda.h>
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

struct Inputs {        // device pointers, layouts as in include/tc.h
  const double *eps, *t1, *t2, *ovvv, *ovoo, *ovov;
};

struct Work {
  const int4 *trip;    // (i, j, k, weight)
  const int4 *orb;     // (P, Q, R, 0) tile indices
  double *partial;     // [n_items][2]: the item's E_(T) part and its E[5]_ST (V r3(W)/D) part
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
// Geometry of one job's split path (tc_split.cu): W-term GEMMs with 128-row M
// tiles over the v^2 virtual pairs, K blocks of 16, N chunks over v.
struct SplitGeom {
  int o, v, S;
  int mt;                // M tiles: ceil(v^2 / 128)
  int kbv, kbo;          // 16-wide blocks over a virtual / an occupied index (kbv sets the N padding)
  int hv, ho;            // 8-wide K halves over a virtual / an occupied index
  int nch, nc;           // N chunks and their width (multiple of 16, <= 256; <= 224 at s = 4)
  int vc;                // innermost extent of the W buffer and FP32 copies (v rounded up to 4)
  int nb;                // triplets per block (capacity of the W buffer)
};
// Byte offsets of the operand images, FP32 copies and W buffer inside a
// job's split workspace.
struct SplitLayout {
  SplitGeom g;
  size_t pa, pa2, hc, hc2, tb, hb, t1f, epsf, ovovf, y;
  size_t total;
};
struct WtJob {           // one job's block of triplets in a W-term launch
  SplitGeom g;
  const int4 *trip;      // the job's triplet table
  int t0, nt;            // triplets [t0, t0 + nt) of the table
  const unsigned char *pa, *pa2, *hc, *hc2, *tb, *hb;
  float *y;              // W buffer [nt][a][b][vc]: W_abc = F(i,j,k)[ab,c] + F(i,k,j)[ac,b] + F(j,k,i)[bc,a]
  int gsel;              // which F this launch forms: 0 F(i,j,k) (stores), 1 F(i,k,j), 2 F(j,k,i) (add)
  long long item0;       // first global item of this job in the launch (set by the launcher)
};
struct WtBatch {
  int njobs;
  int stages, nprod;     // set by the launcher
  size_t slot;           // set by the launcher: stage stride in shared memory
  long long total_items;
  int *err;
  WtJob job[MAX_BATCH];
};
struct EnJob {           // one job's block of triplets in an energy launch
  CUtensorMap ymap;      // 4-D map of the W buffer: (c, b, a, triplet)
  CUtensorMap gmap;      // 5-D map of the FP32 (p u|q w) in both orders
  CUtensorMap tmap;      // 2-D map of the FP32 t1
  Dims d;
  SplitGeom g;
  const int4 *trip, *orb;
  const double *eps;
  const float *t1f;      // t1 [o][vc]
  const float *epsf;     // eps as float pairs: [0, o+v) hi, [o+v, 2(o+v)) lo
  const float *ovovf;    // [2][o][v][o][vc]: (p u|q w) at [0][p][u][q][w] and [1][q][w][p][u]
  const float *y;
  double *partial;       // [n_items][2], slot t * items_per_trip + chunk
  int t0, nt;
  long long item0;
};
struct EnBatch {
  int njobs;
  long long total_items;
  int *err;
  EnJob job[MAX_BATCH];
};
int split_tile();
// Orbits per energy work item of the split path: about 8 items per SM of a
// 152-SM GPU in each energy launch, so the per-item reduction is amortised.
int split_orb_per_item(int o, int v, int S);
SplitGeom split_geom(int o, int v, int S);
SplitLayout split_layout(int o, int v, int S);
// Operand images and FP32 copies of a job: launch_split_prep builds all of
// them; launch_split_prep_common builds those of t1 and the orbital energies
// and launch_split_prep_range those read from t2, ovvv, ovoo and ovov rows
// whose first occupied index lies in [p0, p1) (what a triplet (i, j, k) with
// i >= j >= k reads lies in the rows p <= i).
cudaError_t launch_split_prep(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st);
cudaError_t launch_split_prep_common(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st);
cudaError_t launch_split_prep_range(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st, int p0, int p1);
int split_prep_launches();
int split_prep_range_launches();
WtJob wt_job(const SplitLayout &L, const void *ws, const int4 *trip, int t0, int nt);
// Energy job of triplets [t0, t0 + nt); encodes its tensor map (driver entry point).
cudaError_t en_job(EnJob *out, const Dims &d, const SplitLayout &L, const void *ws, const Inputs &in, const Work &w,
                   int t0, int nt);
// W-term launches per block of triplets: one per F, in the order gsel = 0, 1, 2.
constexpr int SPLIT_WT_LAUNCHES = 3;
// One block of triplets: the three W-term launches, then the energy launch,
// on st.  w0 / w1 (optional) are recorded around the W-term launches.
cudaError_t launch_split_block(WtBatch &wb, EnBatch &eb, int S, int num_sms, cudaStream_t st,
                               cudaEvent_t w0 = nullptr, cudaEvent_t w1 = nullptr);
// Prepare the batches as launch_split_block would and fill the kernel-node
// parameters of its launches: wb[0] is filled by the caller and copied into
// wb[1], wb[2] (gsel 1, 2); wargs[f] / wp[f] belong to wb[f] (f < 3), eargs[0]
// / ep to eb.  The nodes must run in the order wp[0], wp[1], wp[2], ep.
cudaError_t split_block_params(WtBatch *wb, EnBatch &eb, int S, int num_sms, void **wargs, void **eargs,
                               cudaKernelNodeParams *wp, cudaKernelNodeParams *ep);

// ---------------------------------------------------------------- integrals from DF factors (tc_df.cu)
// (ia|bd), (ia|jl) and (ia|jb) from B[nq][o+v][o+v] (Eq. 6) as exact digit
// products on the tensor cores.  scratch: df_scratch_bytes(o, v, nq) device
// bytes.  *digits receives the number of base-256 digits the factors needed
// (at most 7); the call synchronises st once to read it.
size_t df_scratch_bytes(int o, int v, int nq);
cudaError_t df_assemble(const double *B, int nq, int o, int v, double *ovvv, double *ovoo, double *ovov,
                        void *scratch, int num_sms, cudaStream_t st, int *digits);
// Device error flag of the assembly's kernels inside its scratch (0 = fine).
int *df_error_flag(void *scratch, int o, int v, int nq);

// ---------------------------------------------------------------- reduction
struct RedJob {
  int n_trip, items_per_trip, o;
  const int4 *trip;
  const double *partial;
  double *e_trip;        // [n_trip] weighted triplet contributions
  double *e_ijk;         // optional [o][o][o]
  double *out;           // [3]: E, sum |e| and E[5]_ST
};
struct RedBatch {
  int njobs;
  RedJob job[MAX_BATCH];
};
cudaError_t launch_reduce(const RedBatch &b, cudaStream_t st);

}  // namespace tc
