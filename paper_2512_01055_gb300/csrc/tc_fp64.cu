// FP64 path: W (Eqs. 2, 5) built with FP64 tensor-core tiles (mma.sync m8n8k4
// f64), V (Eq. 3), D (Fig. 4 sign) and the bracket of Eq. 1 fused in one
// persistent kernel.  W never leaves shared memory.
//
// One work item = (occupied triplet, chunk of tile orbits); see tc_internal.cuh.
// For every distinct tile block (X, Y, Z) of an orbit the kernel forms
//
//   W^{xyz} = sum over the six permutations u of the positions (0,1,2) of
//       sum_f (o_{u0} g_{u0} | g_{u1} f) t2[o_{u2}][o_{u1}][g_{u2}][f]      (particle, K = v)
//     - sum_l (o_{u0} g_{u0} | o_{u1} l) t2[l][o_{u2}][g_{u1}][g_{u2}]       (hole, K = o)
//
// where (o_0, o_1, o_2) = (i, j, k) and (g_0, g_1, g_2) = (x, y, z): Eq. 2's
// bracket with G_if^ab = (ia|fb) = (ia|bf) (real orbitals) summed over P of
// Eq. 5.  The particle sums are GEMMs whose rows are the pairs (g_{u0}, g_{u1})
// of two tiles and whose columns are g_{u2} of the third; each warp owns one
// 8x8 DMMA tile of each of the six GEMMs.
//
// Epilogue, per canonical point (a >= b >= c) with the six values
// w_s = W^{s(abc)} and v_s = V^{s(abc)}:  the bracket of Eq. 1 at the point
// s(abc) is 3 w_s + S_same - 2 S_other, where S_same / S_other are the sums of
// w over the permutations of the same / opposite parity as s; the point's
// contribution is  sum_s (w_s + v_s) (bracket_s) / D_abc  divided by the number
// of permutations that fix (a, b, c).  Summed over canonical points and
// weighted triplets this is Eq. 1.
#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int NT = 8;            // tile edge
constexpr int NT2 = NT * NT;
constexpr int NT3 = NT2 * NT;
constexpr int KC = 16;           // K chunk of the particle GEMMs
constexpr int LDA = KC + 1;      // padded row length in shared memory
constexpr int THREADS = 256;     // 8 warps: warp w owns GEMM rows 8w .. 8w+7
constexpr int SMEM_DOUBLES = 6 * NT3 + 6 * NT2 * LDA + 6 * NT * LDA;

__device__ __forceinline__ void dmma(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(c[0]), "+d"(c[1]) : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(THREADS, 2)
tc_fp64_kernel(const __grid_constant__ FpBatch B) {
  extern __shared__ double smem[];
  double *Ws = smem;                     // [6][NT3]   W of the orbit's blocks
  double *As = Ws + 6 * NT3;             // [6][NT2][LDA] particle A rows, one set per u
  double *Bs = As + 6 * NT2 * LDA;       // [6][NT][LDA]  particle B rows (t2 panels)
  __shared__ long long s_item;
  __shared__ double s_red[THREADS / 32], s_red5[THREADS / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(B.counter, 1u);
    __syncthreads();
    const long long gitem = s_item;
    if (gitem >= B.total_items) break;
    int jc = 0;                                  // the job owning this global item
    while (jc + 1 < B.njobs && gitem >= B.job[jc + 1].item0) ++jc;
    const Dims &d = B.job[jc].d;
    const Inputs &in = B.job[jc].in;
    const Work &w = B.job[jc].w;
    const long long item = gitem - B.job[jc].item0 + B.job[jc].item_base;
    const int o = d.o, v = d.v;
    const long long vv = (long long)v * v;
    const int t = (int)(item / d.items_per_trip);
    const int chunk = (int)(item % d.items_per_trip);
    const int4 tr = w.trip[t];
    const int occ[3] = {tr.x, tr.y, tr.z};
    double acc = 0.0, acc5 = 0.0;                // E_(T) and its V part E[5]_ST

    const int ob0 = chunk * d.orb_per_item;
    const int ob1 = min(d.n_orb, ob0 + d.orb_per_item);
    for (int ob = ob0; ob < ob1; ++ob) {
      const int4 og = w.orb[ob];
      const int tl[3] = {og.x, og.y, og.z};
      // distinct block holding each formal permutation of the tile triple
      int blk[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        blk[s] = s;
        for (int s2 = 0; s2 < s; ++s2) {
          if (blk[s] == s && tl[perm3(s2, 0)] == tl[perm3(s, 0)] && tl[perm3(s2, 1)] == tl[perm3(s, 1)] &&
              tl[perm3(s2, 2)] == tl[perm3(s, 2)])
            blk[s] = s2;
        }
      }

      for (int s = 0; s < 6; ++s) {
        if (blk[s] != s) continue;
        double *W = Ws + s * NT3;
        const int g0[3] = {tl[perm3(s, 0)] * NT, tl[perm3(s, 1)] * NT, tl[perm3(s, 2)] * NT};

        // ---------------- particle term: six GEMMs, DMMA tiles ----------------
        double c[6][2];
#pragma unroll
        for (int u = 0; u < 6; ++u) c[u][0] = c[u][1] = 0.0;

        for (int f0 = 0; f0 < v; f0 += KC) {
          // stage A rows: As[u][r0*NT + r1][kk] = (o_{u0} g_{u0} | g_{u1} f0+kk)
          for (int e = tid; e < 6 * NT2 * KC; e += THREADS) {
            const int kk = e % KC, r = (e / KC) % NT2, u = e / (KC * NT2);
            const int p0 = perm3(u, 0), p1 = perm3(u, 1);
            const int x0 = g0[p0] + r / NT, x1 = g0[p1] + r % NT, f = f0 + kk;
            double val = 0.0;
            if (x0 < v && x1 < v && f < v)
              val = __ldg(in.ovvv + (((long long)occ[p0] * v + x0) * vv + (long long)x1 * v + f));
            As[(u * NT2 + r) * LDA + kk] = val;
          }
          // stage B rows: Bs[u][col][kk] = t2[o_{u2}][o_{u1}][g_{u2}+col][f0+kk]
          for (int e = tid; e < 6 * NT * KC; e += THREADS) {
            const int kk = e % KC, col = (e / KC) % NT, u = e / (KC * NT);
            const int p1 = perm3(u, 1), p2 = perm3(u, 2);
            const int x2 = g0[p2] + col, f = f0 + kk;
            double val = 0.0;
            if (x2 < v && f < v)
              val = __ldg(in.t2 + ((((long long)occ[p2] * o + occ[p1]) * v + x2) * v + f));
            Bs[(u * NT + col) * LDA + kk] = val;
          }
          __syncthreads();
#pragma unroll
          for (int kk = 0; kk < KC; kk += 4) {
#pragma unroll
            for (int u = 0; u < 6; ++u) {
              const double a = As[(u * NT2 + warp * NT + (lane >> 2)) * LDA + kk + (lane & 3)];
              const double b = Bs[(u * NT + (lane >> 2)) * LDA + kk + (lane & 3)];
              dmma(c[u], a, b);
            }
          }
          __syncthreads();
        }
        // scatter the six GEMM tiles into W: position u0 <- warp, u1 <- row, u2 <- column
#pragma unroll
        for (int u = 0; u < 6; ++u) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            int lc[3];
            lc[perm3(u, 0)] = warp;
            lc[perm3(u, 1)] = lane >> 2;
            lc[perm3(u, 2)] = 2 * (lane & 3) + e;
            const int idx = (lc[0] * NT + lc[1]) * NT + lc[2];
            if (u == 0) W[idx] = c[u][e]; else W[idx] += c[u][e];
          }
          __syncthreads();
        }

        // ---------------- hole term (K = o), one thread per point ----------------
        for (int q = tid; q < NT3; q += THREADS) {
          const int gg[3] = {g0[0] + q / NT2, g0[1] + (q / NT) % NT, g0[2] + q % NT};
          if (gg[0] >= v || gg[1] >= v || gg[2] >= v) continue;
          double h = 0.0;
#pragma unroll
          for (int u = 0; u < 6; ++u) {
            const int p0 = perm3(u, 0), p1 = perm3(u, 1), p2 = perm3(u, 2);
            const double *G = in.ovoo + (((long long)occ[p0] * v + gg[p0]) * o + occ[p1]) * o;   // (x p|y l), l fastest
            const double *T = in.t2 + ((long long)occ[p2] * v + gg[p1]) * v + gg[p2];           // t2[l][z][q][r]
            const long long lstride = (long long)o * vv;
            for (int l = 0; l < o; ++l) h = fma(__ldg(G + l), __ldg(T + l * lstride), h);
          }
          W[q] -= h;
        }
      }
      __syncthreads();

      // ---------------- energy epilogue over canonical points ----------------
      const double eijk = __ldg(in.eps + occ[0]) + __ldg(in.eps + occ[1]) + __ldg(in.eps + occ[2]);
      for (int q = tid; q < NT3; q += THREADS) {
        const int l3[3] = {q / NT2, (q / NT) % NT, q % NT};
        const int g[3] = {tl[0] * NT + l3[0], tl[1] * NT + l3[1], tl[2] * NT + l3[2]};
        if (g[0] >= v || g[1] >= v || g[2] >= v) continue;
        if (g[0] < g[1] || g[1] < g[2]) continue;
        double ws[6], vs[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          const int p0 = perm3(s, 0), p1 = perm3(s, 1), p2 = perm3(s, 2);
          ws[s] = Ws[blk[s] * NT3 + (l3[p0] * NT + l3[p1]) * NT + l3[p2]];
          const int x = g[p0], y = g[p1], z = g[p2];
          // V^{xyz} = t_i^x (jy|kz) + t_j^y (ix|kz) + t_k^z (ix|jy)
          const double *ov = in.ovov;
          vs[s] = __ldg(in.t1 + occ[0] * v + x) * __ldg(ov + (((long long)occ[1] * v + y) * o + occ[2]) * v + z)
                + __ldg(in.t1 + occ[1] * v + y) * __ldg(ov + (((long long)occ[0] * v + x) * o + occ[2]) * v + z)
                + __ldg(in.t1 + occ[2] * v + z) * __ldg(ov + (((long long)occ[0] * v + x) * o + occ[1]) * v + y);
        }
        const double se = ws[0] + ws[3] + ws[4];
        const double so = ws[1] + ws[2] + ws[5];
        double sum = 0.0, sum5 = 0.0;
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          const double br = 3.0 * ws[s] + (perm3_even(s) ? se - 2.0 * so : so - 2.0 * se);
          sum = fma(ws[s] + vs[s], br, sum);
          sum5 = fma(vs[s], br, sum5);
        }
        const double D = eijk - (__ldg(in.eps + o + g[0]) + __ldg(in.eps + o + g[1]) + __ldg(in.eps + o + g[2]));
        const double mult = (g[0] == g[2]) ? 6.0 : ((g[0] == g[1] || g[1] == g[2]) ? 2.0 : 1.0);
        const double rdm = 1.0 / (D * mult);
        acc = fma(sum, rdm, acc);
        acc5 = fma(sum5, rdm, acc5);
      }
      __syncthreads();
    }

    // block reduction of the item's partial (fixed order -> deterministic)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc += __shfl_down_sync(0xffffffffu, acc, off);
      acc5 += __shfl_down_sync(0xffffffffu, acc5, off);
    }
    if (lane == 0) { s_red[warp] = acc; s_red5[warp] = acc5; }
    __syncthreads();
    if (tid == 0) {
      double s = 0.0, s5 = 0.0;
      for (int i2 = 0; i2 < THREADS / 32; ++i2) { s += s_red[i2]; s5 += s_red5[i2]; }
      w.partial[2 * item] = s;
      w.partial[2 * item + 1] = s5;
    }
    __syncthreads();
  }
}

}  // namespace

int fp64_tile() { return NT; }
size_t fp64_smem_bytes() { return sizeof(double) * (size_t)SMEM_DOUBLES; }

// The dynamic shared-memory limit is a per-device attribute of the kernel and
// exceeds the 48 KB default, so it is set on the current device before every
// occupancy query and launch (a cheap host-side call; no process-wide flag
// that would skip it on a second device).
static cudaError_t configure() {
  return cudaFuncSetAttribute(tc_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fp64_smem_bytes());
}

cudaError_t fp64_blocks_per_sm(int *n) {
  cudaError_t e = configure();
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, tc_fp64_kernel, THREADS, fp64_smem_bytes());
  if (e == cudaSuccess && *n < 1) *n = 1;
  return e;
}

void fp64_node_params(const FpBatch &b, int grid, void **args, cudaKernelNodeParams *p) {
  args[0] = (void *)&b;
  *p = cudaKernelNodeParams{};
  p->func = (void *)tc_fp64_kernel;
  p->gridDim = dim3(grid);
  p->blockDim = dim3(THREADS);
  p->sharedMemBytes = (unsigned)fp64_smem_bytes();
  p->kernelParams = args;
}

cudaError_t launch_fp64(const FpBatch &b, int grid, cudaStream_t st) {
  cudaError_t e = configure();
  if (e != cudaSuccess) return e;
  tc_fp64_kernel<<<grid, THREADS, fp64_smem_bytes(), st>>>(b);
  return cudaGetLastError();
}

}  // namespace tc
