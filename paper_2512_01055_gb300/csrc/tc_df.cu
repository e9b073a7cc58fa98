// Integral blocks from density-fitting (or Cholesky) factors on the tensor
// cores (Eq. 6 of the paper: (pq|rs) = sum_Q B_pq^Q B_rs^Q):
//   ovvv[i][a][b][d] = sum_Q B[Q][i][o+a] B[Q][o+b][o+d]
//   ovoo[i][a][j][l] = sum_Q B[Q][i][o+a] B[Q][j][l]
//   ovov[i][a][j][b] = sum_Q B[Q][i][o+a] B[Q][j][o+b]
// Each block is a product C[m][n] = sum_Q X[Q][m] Y[Q][n] of two "operands",
// strided views of B with rows m (resp. n) and K = Q.
//
// Exact digit products.  Every operand row r gets a power-of-two scale 2^e_r
// with |x| < 2^e_r over its K values, and each value becomes P signed base-256
// digits of x 2^-e_r:  x = 2^e_r sum_p d_p 2^(-8(p+1)) (+ a tail below
// 2^(e_r - 8P - 1) when P < 7 does not reach the last bit).  d_0 lies in
// [-256, 256], the others in [-128, 128]: integers that BF16 holds exactly.
// So x y = 2^(e_m + e_n) sum_(p,q) d_p d'_q 2^(-8(p+q+2)), and the digit
// products of one class w = p + q share a weight.  The tensor cores multiply
// digits exactly and sum each class in FP32 (TMEM) over chunks of K short
// enough that every partial sum is an integer below 2^24, so each chunk's
// class sums S_w are exact; the drain converts them to integers and adds
// H = S_0 2^16 + S_1 2^8 + S_2 and L = S_3 2^24 + S_4 2^16 + S_5 2^8 + S_6
// over the chunks in 64-bit integers (exact), and finally
//   C = 2^(e_m + e_n - 32) H + 2^(e_m + e_n - 64) L
// with one rounding.  P is the number of digits that the inputs need (found
// on the device, at most 7): factors on a 2^-20 grid need 3 and then every
// integral comes out exact, bit for bit what any exact summation gives;
// general FP64 factors take 7 digits and pairs with p + q <= 6, which leaves
// an error far below the FP64 rounding of a dot product of length Q.
//
// GEMM kernel: one persistent CTA per SM walks 128 x 64 output tiles.  Warps 0
// and 1 copy the digit images of a K block (both operands, all P digits, two
// 8-wide K halves) into a ring of shared-memory stages with cp.async.bulk;
// warp 2 owns TMEM (7 classes x 64 columns) and its lane 0 issues one
// tcgen05.mma (M = 128, N = 64, K = 16) per digit pair and K block; warps
// 4-19 drain each chunk's class sums (warp w: TMEM lanes 32 (w % 4) .. +31,
// 16 of the 64 columns) into their 64-bit sums and, after the tile's last
// chunk, write the FP64 results.  Every mbarrier wait is bounded.
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>

#include "tc_internal.cuh"
#include "tc_ptx.cuh"

namespace tc {
namespace {

constexpr int DF_PMAX = 7;            // most digits per value
constexpr int DF_WMAX = 7;            // digit-pair classes kept (w = p + q <= 6)
constexpr int DF_MROWS = 128;         // output tile rows (A operand)
constexpr int DF_NCOLS = 64;          // output tile columns (B operand)
constexpr int DF_THREADS = 640;       // 20 warps
constexpr int DF_DRAIN_WARP0 = 4;
constexpr int DF_DRAIN_THREADS = 512;
constexpr int DF_NPROD = 2;
constexpr int DF_MAX_STAGES = 8;
constexpr int DF_SMEM_MAX = 232448 - 4096;
constexpr int DF_ERR_FULL = 21, DF_ERR_EMPTY = 22, DF_ERR_ACCFULL = 23, DF_ERR_ACCEMPTY = 24, DF_ERR_TEARDOWN = 25;

// A strided view of B[Q][n][n] (n = o + v) as rows r in [0, rows) over K = Q:
// element (Q, r) = B[Q][row0 + r / cols][col0 + r % cols].
struct DfOperand {
  int row0, col0, cols;
  long long rows;
};

__device__ __forceinline__ double df_elem(const double *B, int n, const DfOperand &op, int q, long long r) {
  const long long br = op.row0 + r / op.cols, bc = op.col0 + r % op.cols;
  return B[((long long)q * n + br) * n + bc];
}

// Row scales: e[r] such that every |element (Q, r)| < 2^e[r] (0 for a zero row).
__global__ void df_scales(const double *__restrict__ B, int n, int nq, DfOperand op, int *__restrict__ e) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < op.rows; r += (long long)gridDim.x * blockDim.x) {
    double mx = 0.0;
    for (int q = 0; q < nq; ++q) mx = fmax(mx, fabs(df_elem(B, n, op, q, r)));
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);            // mx = f 2^ex, f in [0.5, 1)
    e[r] = ex;
  }
}

// The base-256 digits of x 2^-e (|x 2^-e| < 1); returns the number of digits
// up to the last nonzero one (0 for x = 0).
__device__ __forceinline__ int df_digits(double x, int e, double (&d)[DF_PMAX]) {
  double t = ldexp(x, -e);
  int used = 0;
#pragma unroll
  for (int p = 0; p < DF_PMAX; ++p) {
    t *= 256.0;                              // exact: a power of two
    d[p] = rint(t);
    t -= d[p];                               // exact: |t| < 2^8 and d[p] is t rounded to an integer
    if (d[p] != 0.0) used = p + 1;
  }
  return used;
}

// Largest number of digits any element of the operand needs (atomic max).
__global__ void df_digit_count(const double *__restrict__ B, int n, int nq, DfOperand op, const int *__restrict__ e,
                               int *__restrict__ pmax) {
  int mine = 0;
  const long long total = op.rows * nq;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % op.rows;
    const int q = (int)(t / op.rows);
    double d[DF_PMAX];
    mine = max(mine, df_digits(df_elem(B, n, op, q, r), e[r], d));
  }
  for (int off = 16; off > 0; off >>= 1) mine = max(mine, __shfl_xor_sync(0xffffffffu, mine, off));
  if ((threadIdx.x & 31) == 0 && mine > 0) atomicMax(pmax, mine);
}

// Digit image of an operand in the tensor core's K-major no-swizzle layout:
// [row tile][K block][half][digit][R rows][8 BF16], core matrices of 8 rows x
// 16 bytes, 8-row groups 128 bytes apart.  One thread per (tile, K block,
// half, row) converts 8 K values; rows past op.rows and Q past nq are zero.
__global__ void df_image(const double *__restrict__ B, int n, int nq, DfOperand op, const int *__restrict__ e, int P,
                         int R, int nkb, long long ntiles, unsigned char *__restrict__ out) {
  const long long total = ntiles * nkb * 2 * R;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int row = (int)(t % R);
    const long long hb = t / R;              // (tile, K block, half)
    const int half = (int)(hb & 1);
    const int kb = (int)((hb >> 1) % nkb);
    const long long tile = (hb >> 1) / nkb;
    const long long r = tile * R + row;
    const int q0 = kb * 16 + half * 8;
    __align__(16) __nv_bfloat16 dig[DF_PMAX][8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double d[DF_PMAX];
      const int q = q0 + u;
      const double x = (r < op.rows && q < nq) ? df_elem(B, n, op, q, r) : 0.0;
      df_digits(x, r < op.rows ? e[r] : 0, d);
#pragma unroll
      for (int p = 0; p < DF_PMAX; ++p) dig[p][u] = __double2bfloat16(d[p]);   // integers |d| <= 256: exact
    }
    unsigned char *base = out + (size_t)hb * P * R * 16 + (row >> 3) * 128 + (row & 7) * 16;
    for (int p = 0; p < P; ++p) *(uint4 *)(base + (size_t)p * R * 16) = *(const uint4 *)dig[p];
  }
}

// One product C[m][n] = sum_Q X[Q][m] Y[Q][n] (see the file comment).
struct DfGemm {
  const unsigned char *a, *b;     // digit images of X (128-row tiles) and Y (64-row tiles)
  const int *ea, *eb;             // row scales
  double *c;
  long long M, N, ldc;
  int mt, nt;                     // tiles of 128 rows, 64 columns
  int nkb;                        // K blocks of 16
  int P;                          // digits per value
  int W;                          // classes kept: min(2P - 1, 7)
  int kc;                         // K blocks per chunk (class sums stay below 2^24)
  int stages;
  size_t slot;                    // stage bytes: 2 P (2048 + 64 x 16)
  int *err;
};

__device__ __forceinline__ void df_bar_drain() { asm volatile("bar.sync 1, %0;" :: "n"(DF_DRAIN_THREADS) : "memory"); }
__device__ __forceinline__ void df_bar_prod() { asm volatile("bar.sync 2, %0;" :: "n"(DF_NPROD * 32) : "memory"); }

// Tile t -> (m tile, n tile), in groups of 16 m tiles so that the CTAs working
// at the same time share their operands' tiles through L2.
__device__ __forceinline__ void df_tile(const DfGemm &G, long long t, int &mt, int &nt) {
  constexpr int GROUP = 16;
  const long long per_group = (long long)GROUP * G.nt;
  const long long g = t / per_group;
  const int first = (int)(g * GROUP);
  const int rows = min(GROUP, G.mt - first);
  const long long in = t - g * per_group;
  mt = first + (int)(in % rows);
  nt = (int)(in / rows);
}

__device__ __forceinline__ void df_mma(uint32_t dcol, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(dcol), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void df_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(DF_THREADS, 1) df_gemm_kernel(const __grid_constant__ DfGemm G) {
  extern __shared__ __align__(1024) unsigned char df_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)df_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[DF_MAX_STAGES], empty_bar[DF_MAX_STAGES];
  __shared__ __align__(8) uint64_t accfull_bar, accempty_bar, teardown_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ int drain_ok;
  __shared__ long long last_seq[DF_NPROD][DF_MAX_STAGES];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = (long long)G.mt * G.nt;
  const int nchunk = (G.nkb + G.kc - 1) / G.kc;
  const uint32_t abytes = 2u * G.P * DF_MROWS * 16, bbytes = 2u * G.P * DF_NCOLS * 16;

  if (tid < DF_NPROD * DF_MAX_STAGES) last_seq[tid / DF_MAX_STAGES][tid % DF_MAX_STAGES] = -1;
  if (tid == 0) {
    for (int s = 0; s < G.stages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&accfull_bar, 1);
    mbar_init(&accempty_bar, 1);
    mbar_init(&teardown_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base_sh;

  if (warp < DF_NPROD) {
    // ------------------------------------------------ producers: one K block per stage
    const int pw = warp;
    int stage = 0, rr = 0;
    uint32_t phase = 0;
    long long seq = 0;
    bool ok = true;
    for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
      int mtile, ntile;
      df_tile(G, t, mtile, ntile);
      for (int kb = 0; kb < G.nkb; ++kb, ++seq) {
        const bool mine = rr == pw;
        if (++rr == DF_NPROD) rr = 0;
        if (mine) {
          int got = 1;
          if (lane == 0) {
            got = mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, G.err, DF_ERR_EMPTY) ? 1 : 0;
            if (got) {
              last_seq[pw][stage] = seq;
              mbar_expect_tx(&full_bar[stage], abytes + bbytes);
            }
          }
          got = __shfl_sync(0xffffffffu, got, 0);
          if (!got) { ok = false; break; }
          unsigned char *sA = sm + (size_t)stage * G.slot, *sB = sA + abytes;
          if (lane == 0) bulk_load(sA, G.a + ((size_t)mtile * G.nkb + kb) * abytes, abytes, &full_bar[stage]);
          else if (lane == 1) bulk_load(sB, G.b + ((size_t)ntile * G.nkb + kb) * bbytes, bbytes, &full_bar[stage]);
          __syncwarp();
        }
        if (++stage == G.stages) { stage = 0; phase ^= 1u; }
      }
    }
    // every issued copy lands before the CTA may exit: only the latest copy
    // into each stage can still be in flight
    df_bar_prod();
    if (pw == 0 && lane == 0) {
      for (int s = 0; s < G.stages; ++s) {
        long long last = -1;
        for (int q = 0; q < DF_NPROD; ++q) last = max(last, last_seq[q][s]);
        if (last < 0) continue;
        const uint32_t par = (uint32_t)((last / G.stages) & 1);
        const uint32_t a = smem_u32(&full_bar[s]);
        for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, par); ++it) {
          if ((it & 255) == 255) __nanosleep(128);
          if (it == WAIT_LIMIT - 1) atomicCAS(G.err, 0, DF_ERR_TEARDOWN);
        }
      }
    }
    __syncwarp();
  } else if (warp == 2) {
    // ------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc(DF_MROWS, DF_NCOLS);
      const uint32_t alb = (uint32_t)G.P * DF_MROWS * 16, blb = (uint32_t)G.P * DF_NCOLS * 16;   // second K half
      int stage = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        for (int ch = 0; ok && ch < nchunk; ++ch) {
          // the class sums go back from the drain before a chunk starts
          if (!mbar_wait(&accempty_bar, aphase ^ 1u, &abort_flag, G.err, DF_ERR_ACCEMPTY)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int kb0 = ch * G.kc, kb1 = min(G.nkb, kb0 + G.kc);
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full_bar[stage], phase, &abort_flag, G.err, DF_ERR_FULL)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = smem_u32(sm + (size_t)stage * G.slot), sB = sA + (uint32_t)(2 * alb);
            for (int p = 0; p < G.P; ++p)
              for (int q = 0; q < G.P; ++q) {
                const int w = p + q;
                if (w >= G.W) continue;
                // the chunk's first product of class w (smallest p with q < P) starts its sum
                const uint32_t acc = (kb == kb0 && p == max(0, w - (G.P - 1))) ? 0u : 1u;
                df_mma(tbase + (uint32_t)(w * DF_NCOLS), sdesc(sA + p * DF_MROWS * 16, alb),
                       sdesc(sB + q * DF_NCOLS * 16, blb), id, acc);
              }
            df_commit(&empty_bar[stage]);
            if (++stage == G.stages) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          df_commit(&accfull_bar);
          aphase ^= 1u;
        }
      }
      df_commit(&teardown_bar);
      const uint32_t a = smem_u32(&teardown_bar);
      for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, 0); ++it) {
        if ((it & 255) == 255) __nanosleep(128);
        if (it == WAIT_LIMIT - 1) atomicCAS(G.err, 0, DF_ERR_TEARDOWN);
      }
    }
    __syncwarp();
  } else if (warp >= DF_DRAIN_WARP0) {
    // ------------------------------------------------ drain: class sums -> 64-bit sums -> FP64
    const int dw = warp - DF_DRAIN_WARP0;            // 0 .. 15
    const int quarter = warp & 3;                    // TMEM lanes this warp may read
    const int cg = dw >> 2;                          // which 16 of the 64 columns
    const int lrow = 32 * quarter + lane;
    const uint32_t trow = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(cg * 16);
    const int et = tid - DF_DRAIN_WARP0 * 32;
    uint32_t aphase = 0;
    bool ok = true;
    for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
      long long H[16], L[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) H[j] = L[j] = 0;
      for (int ch = 0; ch < nchunk; ++ch) {
        if (et == 0) drain_ok = mbar_wait(&accfull_bar, aphase, &abort_flag, G.err, DF_ERR_ACCFULL) ? 1 : 0;
        df_bar_drain();
        if (!drain_ok) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int w = 0; w < DF_WMAX; ++w) {
          if (w >= G.W) break;
          float s[16];
          tmem_ld16(trow + (uint32_t)(w * DF_NCOLS), s);
          tmem_wait_ld();
          // S_w is an integer below 2^24: exact in FP32 and in int
          const int sh = w < 3 ? 8 * (2 - w) : 8 * (6 - w);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const long long x = (long long)__float2int_rn(s[j]) << sh;
            if (w < 3) H[j] += x;
            else L[j] += x;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        df_bar_drain();
        if (et == 0) mbar_arrive(&accempty_bar);
        aphase ^= 1u;
      }
      if (!ok) break;
      int mtile, ntile;
      df_tile(G, t, mtile, ntile);
      const long long m = (long long)mtile * DF_MROWS + lrow;
      if (m < G.M) {
        const int em = G.ea[m];
        double *crow = G.c + m * G.ldc;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const long long nn = (long long)ntile * DF_NCOLS + cg * 16 + j;
          if (nn < G.N) {
            const int ex = em + G.eb[nn];
            crow[nn] = ldexp((double)H[j], ex - 32) + ldexp((double)L[j], ex - 64);
          }
        }
      }
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512));
  }
}

// Largest |sum over one K value| of a class of digit products, for P digits.
long long df_class_bound(int P) {
  long long best = 0;
  for (int w = 0; w < std::min(2 * P - 1, DF_WMAX); ++w) {
    long long s = 0;
    for (int p = 0; p < P; ++p) {
      const int q = w - p;
      if (q < 0 || q >= P) continue;
      s += (long long)(p == 0 ? 256 : 128) * (q == 0 ? 256 : 128);
    }
    best = std::max(best, s);
  }
  return best;
}

struct DfPlan {
  int o, v, nq, n, nkb;
  DfOperand X, Yvv, Yoo;
  long long mtX, ntX, ntVV, ntOO;   // 128-row tiles of X; 64-row tiles of X, Yvv, Yoo
  size_t e_x, e_vv, e_oo, pmax, err, img_x128, img_x64, img_vv, img_oo, total;
};

size_t img_bytes(long long tiles, int nkb, int P, int R) { return (size_t)tiles * nkb * 2 * P * R * 16; }

DfPlan df_plan(int o, int v, int nq, int P) {
  DfPlan L{};
  L.o = o;
  L.v = v;
  L.nq = nq;
  L.n = o + v;
  L.nkb = (nq + 15) / 16;
  L.X = DfOperand{0, o, v, (long long)o * v};          // (i, a): B[Q][i][o + a]
  L.Yvv = DfOperand{o, o, v, (long long)v * v};        // (b, d): B[Q][o + b][o + d]
  L.Yoo = DfOperand{0, 0, o, (long long)o * o};        // (j, l): B[Q][j][l]
  L.mtX = (L.X.rows + DF_MROWS - 1) / DF_MROWS;
  L.ntX = (L.X.rows + DF_NCOLS - 1) / DF_NCOLS;
  L.ntVV = (L.Yvv.rows + DF_NCOLS - 1) / DF_NCOLS;
  L.ntOO = (L.Yoo.rows + DF_NCOLS - 1) / DF_NCOLS;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = (off + bytes + 255) & ~(size_t)255; return r; };
  L.e_x = take(sizeof(int) * (size_t)L.X.rows);
  L.e_vv = take(sizeof(int) * (size_t)L.Yvv.rows);
  L.e_oo = take(sizeof(int) * (size_t)L.Yoo.rows);
  L.pmax = take(sizeof(int));
  L.err = take(sizeof(int));
  L.img_x128 = take(img_bytes(L.mtX, L.nkb, P, DF_MROWS));
  L.img_x64 = take(img_bytes(L.ntX, L.nkb, P, DF_NCOLS));
  L.img_vv = take(img_bytes(L.ntVV, L.nkb, P, DF_NCOLS));
  L.img_oo = take(img_bytes(L.ntOO, L.nkb, P, DF_NCOLS));
  L.total = off;
  return L;
}

cudaError_t df_gemm(const DfGemm &G0, int num_sms, cudaStream_t st) {
  DfGemm G = G0;
  G.slot = (size_t)2 * G.P * (DF_MROWS + DF_NCOLS) * 16;
  G.stages = (int)std::min<long long>(DF_MAX_STAGES, (long long)(DF_SMEM_MAX - 1024) / (long long)G.slot);
  if (G.stages < DF_NPROD) return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)G.stages * G.slot;
  cudaError_t e = cudaFuncSetAttribute(df_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)G.mt * G.nt;
  const int grid = (int)std::max<long long>(1, std::min<long long>(num_sms, tiles));
  df_gemm_kernel<<<grid, DF_THREADS, smem, st>>>(G);
  return cudaGetLastError();
}

}  // namespace

size_t df_scratch_bytes(int o, int v, int nq) { return df_plan(o, v, nq, DF_PMAX).total; }

cudaError_t df_assemble(const double *B, int nq, int o, int v, double *ovvv, double *ovoo, double *ovov, void *scratch,
                        int num_sms, cudaStream_t st, int *digits) {
  const DfPlan L7 = df_plan(o, v, nq, DF_PMAX);       // scales and counters sit where every plan puts them
  unsigned char *base = (unsigned char *)scratch;
  int *e_x = (int *)(base + L7.e_x), *e_vv = (int *)(base + L7.e_vv), *e_oo = (int *)(base + L7.e_oo);
  int *pmax = (int *)(base + L7.pmax), *err = (int *)(base + L7.err);
  const int blocks = num_sms * 8, thr = 256;
  cudaError_t e;
  df_scales<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.X, e_x);
  df_scales<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.Yvv, e_vv);
  df_scales<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.Yoo, e_oo);
  if ((e = cudaMemsetAsync(pmax, 0, 2 * 256, st)) != cudaSuccess) return e;   // pmax and err
  df_digit_count<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.X, e_x, pmax);
  df_digit_count<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.Yvv, e_vv, pmax);
  df_digit_count<<<blocks, thr, 0, st>>>(B, L7.n, nq, L7.Yoo, e_oo, pmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int P = 0;
  if ((e = cudaMemcpyAsync(&P, pmax, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  P = std::max(1, std::min(P, DF_PMAX));
  *digits = P;
  const DfPlan L = df_plan(o, v, nq, P);
  unsigned char *ix128 = base + L.img_x128, *ix64 = base + L.img_x64, *ivv = base + L.img_vv, *ioo = base + L.img_oo;
  df_image<<<blocks, thr, 0, st>>>(B, L.n, nq, L.X, e_x, P, DF_MROWS, L.nkb, L.mtX, ix128);
  df_image<<<blocks, thr, 0, st>>>(B, L.n, nq, L.X, e_x, P, DF_NCOLS, L.nkb, L.ntX, ix64);
  df_image<<<blocks, thr, 0, st>>>(B, L.n, nq, L.Yvv, e_vv, P, DF_NCOLS, L.nkb, L.ntVV, ivv);
  df_image<<<blocks, thr, 0, st>>>(B, L.n, nq, L.Yoo, e_oo, P, DF_NCOLS, L.nkb, L.ntOO, ioo);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  DfGemm G{};
  G.P = P;
  G.W = std::min(2 * P - 1, DF_WMAX);
  G.kc = (int)std::max<long long>(1, ((1LL << 24) - 1) / (16 * df_class_bound(P)));
  G.nkb = L.nkb;
  G.err = err;
  G.a = ix128;
  G.ea = e_x;
  G.M = L.X.rows;
  G.mt = (int)L.mtX;
  // (ia|bd): rows (i, a), columns (b, d)
  G.b = ivv; G.eb = e_vv; G.c = ovvv; G.N = L.Yvv.rows; G.ldc = G.N; G.nt = (int)L.ntVV;
  if ((e = df_gemm(G, num_sms, st)) != cudaSuccess) return e;
  // (ia|jl): columns (j, l)
  G.b = ioo; G.eb = e_oo; G.c = ovoo; G.N = L.Yoo.rows; G.ldc = G.N; G.nt = (int)L.ntOO;
  if ((e = df_gemm(G, num_sms, st)) != cudaSuccess) return e;
  // (ia|jb): columns (j, b)
  G.b = ix64; G.eb = e_x; G.c = ovov; G.N = L.X.rows; G.ldc = G.N; G.nt = (int)L.ntX;
  return df_gemm(G, num_sms, st);
}

int *df_error_flag(void *scratch, int o, int v, int nq) {
  return (int *)((unsigned char *)scratch + df_plan(o, v, nq, DF_PMAX).err);
}

}  // namespace tc
