// Split-precision path: W (Eqs. 2, 5) from BF16 slices on the tcgen05 tensor
// cores (FP32 accumulation in TMEM), V (Eq. 3) and the Eq. 1 bracket in FP32;
// D (Fig. 4 sign), its reciprocal, each point's quotient and the sums over a
// work item in float pairs (about 48 significant bits, the FP64-class
// arithmetic of GB300's FP32 pipes); item partials in FP64.
//
// Slices.  Every FP64 operand x is written as s BF16 numbers x_0 + ... + x_{s-1}
// with x_0 = bf16(x) and x_p = bf16(x - x_0 - ... - x_{p-1}) (round to
// nearest; the FP64 residual is exact), the splitting used to emulate higher
// precision with BF16 products (Henry, Tang, Heinecke, ARITH 2019).  A product
// is approximated by the slice pairs (p, q) with p + q < s.
//
// W as three GEMMs per triplet.  For one occupied triplet (i, j, k), the six
// terms X of Eq. 5 regroup by the virtual index that the t2 factor of the
// particle product (and the integral of the hole product) carries:
//   W_abc = F(i,j,k)[ab, c] + F(i,k,j)[ac, b] + F(j,k,i)[bc, a]
//   F(p,q,r)[xy, z] =   sum_f G_pf^xy t_rq^zf + sum_f G_qf^yx t_rp^zf
//                     - sum_l t_lp^yx G_rq^zl - sum_l t_lq^xy G_rp^zl
// (G_pq^rs = (pr|qs)).  F(i,j,k) holds the particle parts of X(ijk,abc) and
// X(jik,bac) and the hole parts of X(kji,cba) and X(kij,cab); F(i,k,j) and
// F(j,k,i) hold the other four pairs.  Each F is one GEMM with M = v^2 row
// pairs (x, y), N = v and K = 2v + 2o (four segments), so the tensor cores run
// with N up to 256 instead of the 16-wide panels a tile-local W would allow.
//
// W-term kernel.  One launch forms one F for a block of triplets; a work item
// is (128-row M tile, triplet, N chunk), M-tile-major so the triplets of the
// launch share A tiles through L2.
// Per K block of 16 the MMA warp issues one MMA per slice pair: level 0 into
// accumulator L0, levels >= 1 into L1 (TMEM columns [0, nc) and [nc, 2nc)).
// The FP32 accumulation along K rounds systematically, so L0 is restarted
// every KCHAIN blocks (256 K values): the drain warps (a thread holds one tile
// row, half its columns) add each finished chain into the row's FP32 sum in
// registers; on the last chain they add L1 and write the row, in [a][b][c]
// orientation, into the job's W buffer Y[triplet][a][b][c].  While the drain
// reads a finished chain's L0, the MMA warp issues the L1 products of the next
// chain's first DEFER K blocks and only then their level-0 products.  The three F
// launches of a block run in order: the first stores, the other two add their
// rows to the stored values (L2 reductions), so Y ends as W with each
// element's three contributions added in one fixed order.  Shared memory holds only the
// operand pipeline.
//
// Energy kernel.  A work item is (triplet, chunk of tile orbits) as in the
// FP64 path.  Per orbit it loads the six 16^3 W blocks (TMA) into shared
// memory and evaluates the Eq. 1 bracket at the orbit's canonical points,
// writing FP64 partials (E_(T) and its V part) per item.
//
// Operand images.  The slicer writes the operands directly in the tensor
// core's K-major no-swizzle layout as a sequence of 8-wide K halves: a half is
// the s slices of rows x 16 bytes (8-row x 16-byte core matrices, 8-row groups
// 128 bytes apart).  A K block of 16 is two halves, s slices apart in shared
// memory (the descriptor's leading byte offset), so a block may take its
// halves from two segments and a segment is padded to 8 K values, not 16.  A
// pipeline stage is two contiguous bulk copies (cp.async.bulk), the A halves
// and the B halves, or four when the block spans a segment boundary.
//
// Warp roles of the W-term kernel (384 threads): warps 0, 10 and 11 issue the
// bulk copies (a warp completes about one stage per ~0.37 us, several warps
// overlap), warp 1 owns TMEM and lane 0 issues the MMAs, warps 2-9 drain TMEM
// (warp w reads TMEM lanes 32 (w % 4) .. +31, half the columns each).
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// lets every role leave its loop, waits (bounded) for its own copies and MMAs
// and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "tc_internal.cuh"
#include "tc_ptx.cuh"

namespace tc {
namespace {

constexpr int NT = 16;                    // virtual tile edge of the energy orbits
constexpr int KB = 16;                    // K values per block (one MMA)
constexpr int MROWS = 128;                // rows of an M tile
constexpr int A_BLK = MROWS * KB * 2;     // bytes of one A slice block
constexpr int A_HALF = MROWS * 16;        // bytes of one A slice half (8 K values)
constexpr int NCMAX = 256;                // widest N chunk: two accumulators of 256 columns fill TMEM
constexpr int NCMAX_S4 = 224;             // widest N chunk at s = 4, where more than DEFER stages must fit
constexpr int NC_NARROW = 224;            // chunks up to this width: at most 7 column groups per drain thread
constexpr int MAXS = 4;
constexpr int MAX_STAGES = 8;
constexpr int NPROD = 3;
constexpr int THREADS = 384;
constexpr int DRAIN_THREADS = 256;
constexpr int SMEM_DYN_MAX = 232448 - 2048;  // opt-in limit minus static shared memory and slack
// Longest run of K blocks accumulated in one tensor-core accumulator (see above).
constexpr int KCHAIN = 16;
// K blocks of a later chain whose level-0 products wait for the drain to free
// L0 while their higher-level products already run (fewer than the stages).
constexpr int DEFER = 4;

constexpr int ERR_TIMEOUT_FULL = 11, ERR_TIMEOUT_EMPTY = 12, ERR_TIMEOUT_ACCFULL = 13,
              ERR_TIMEOUT_ACCEMPTY = 14, ERR_TIMEOUT_TEARDOWN = 15;

// energy kernel
constexpr int EN_CONSUMERS = 512;        // copy + compute threads
constexpr int EN_WARPS = EN_CONSUMERS / 32;
constexpr int EN_THREADS = EN_CONSUMERS + 32;   // plus one warp that walks the work and issues the TMA loads
constexpr int BOXF = NT * NT * NT;        // floats of a 16^3 box
constexpr int EN_SLOTS = 5;               // W staging slots (one box each)
constexpr int EN_VSETS = 2;               // V sets (one orbit's G and t1 tiles each)
constexpr int WX = 273, WY = 17;          // W block index = x*WX + y*WY + z (bank-friendly)
constexpr int WBLK = 4368;                // floats per W block (>= 15*WX + 15*WY + 16)
// An orbit's V set: 18 G tiles of 16 x 16 and 9 t1 rows of 16 (each t1 row at
// a 128-byte TMA destination)
constexpr int G_FLOATS = 18 * NT * NT;
constexpr int T1_ROW = 32;
constexpr int GSET_FLOATS = G_FLOATS + 9 * T1_ROW;
constexpr int GSET_TX = (G_FLOATS + 9 * NT) * 4;   // bytes the TMA delivers per set
constexpr int EN_SMEM = 1024 + (EN_SLOTS * BOXF + EN_VSETS * GSET_FLOATS + 6 * WBLK) * 4;
static_assert(EN_SMEM + 1024 <= 232448, "energy kernel shared memory");

__device__ __forceinline__ void mma_bf16(uint32_t dcol, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(dcol), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void drain_bar() { asm volatile("bar.sync 1, %0;" :: "n"(DRAIN_THREADS) : "memory"); }
__device__ __forceinline__ void prod_bar() { asm volatile("bar.sync 2, %0;" :: "n"(NPROD * 32) : "memory"); }

// Distinct tile block holding each formal permutation of the orbit's tile triple.
__host__ __device__ __forceinline__ void orbit_blocks(const int tl[3], int blk[6]) {
#pragma unroll
  for (int s = 0; s < 6; ++s) {
    blk[s] = s;
    for (int s2 = 0; s2 < s; ++s2)
      if (blk[s] == s && tl[perm3(s2, 0)] == tl[perm3(s, 0)] && tl[perm3(s2, 1)] == tl[perm3(s, 1)] &&
          tl[perm3(s2, 2)] == tl[perm3(s, 2)])
        blk[s] = s2;
  }
}

// ---------------------------------------------------------------- W-term kernel

// Item q of a job -> (M tile, triplet in the block, N chunk), M-tile-major; a
// launch forms one F (J.gsel) for every triplet of the block.
__device__ __forceinline__ void wt_decode(const WtJob &J, long long q, int &m, int &tl, int &g, int &nci) {
  nci = (int)(q % J.g.nch);
  q /= J.g.nch;
  g = J.gsel;
  tl = (int)(q % J.nt);
  m = (int)(q / J.nt);
}

// Occupied indices (p, q, r) of F number g for triplet (i, j, k):
// F(i,j,k), F(i,k,j), F(j,k,i).
__device__ __forceinline__ void wt_occ(const WtJob &J, int tl, int g, int &p, int &q, int &r) {
  const int4 t = J.trip[J.t0 + tl];
  if (g == 0)      { p = t.x; q = t.y; r = t.z; }
  else if (g == 1) { p = t.x; q = t.z; r = t.y; }
  else             { p = t.y; q = t.z; r = t.x; }
}

// Sources of K half h (8 K values) of an item: A half (S slices of 128 rows x
// 16 bytes) and B half (S slices of nc rows x 16 bytes).  Segments, hv halves
// over a virtual index or ho over an occupied one: particle G_p/t_rq, particle
// G_q/t_rp, hole t_.p/G_rq, hole t_.q/G_rp.  seg receives the segment, so the
// caller can tell whether two halves are consecutive in one image.
template <int S>
__device__ __forceinline__ void wt_src(const WtJob &J, int m, int nci, int p, int q, int r, int h, int &seg,
                                       const unsigned char *&a, const unsigned char *&b) {
  const SplitGeom &G = J.g;
  const size_t ahb = (size_t)S * A_HALF, bhb = (size_t)S * G.nc * 16;
  if (h < G.hv) {
    seg = 0;
    a = J.pa + (((size_t)p * G.mt + m) * G.hv + h) * ahb;
    b = J.tb + ((((size_t)r * G.o + q) * G.nch + nci) * G.hv + h) * bhb;
    return;
  }
  h -= G.hv;
  if (h < G.hv) {
    seg = 1;
    a = J.pa2 + (((size_t)q * G.mt + m) * G.hv + h) * ahb;
    b = J.tb + ((((size_t)r * G.o + p) * G.nch + nci) * G.hv + h) * bhb;
    return;
  }
  h -= G.hv;
  if (h < G.ho) {
    seg = 2;
    a = J.hc2 + (((size_t)p * G.mt + m) * G.ho + h) * ahb;
    b = J.hb + ((((size_t)r * G.o + q) * G.nch + nci) * G.ho + h) * bhb;
    return;
  }
  h -= G.ho;
  seg = 3;
  a = J.hc + (((size_t)q * G.mt + m) * G.ho + h) * ahb;
  b = J.hb + ((((size_t)r * G.o + p) * G.nch + nci) * G.ho + h) * bhb;
}

// MG: 16-column groups a drain thread holds, 7 for chunks of up to 224
// columns, 8 up to 256.
template <int S, int MG>
__global__ void __launch_bounds__(THREADS, 1)
tc_wterm_kernel(const __grid_constant__ WtBatch B) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t accfull_bar, accempty_bar, teardown_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ int drain_ok;
  __shared__ long long last_seq[NPROD][MAX_STAGES];   // per producer: its latest copy into each stage

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < NPROD * MAX_STAGES) last_seq[tid / MAX_STAGES][tid % MAX_STAGES] = -1;
  if (tid == 0) {
    for (int s = 0; s < B.stages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&accfull_bar, 1);
    mbar_init(&accempty_bar, 1);
    mbar_init(&teardown_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base_sh;
  // A launch that follows this one programmatically may start its CTAs as SMs
  // free up; it waits for this grid's completion before it touches Y.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (warp == 0 || warp >= 10) {
    // ------------------------------------------------------------ bulk-copy producers
    // Every active producer walks the same sequence of K blocks; producer pw
    // fills the blocks whose sequence number is pw modulo nprod.
    const int pw = warp == 0 ? 0 : warp - 9;
    if (pw < B.nprod) {
      int stage = 0, rr = 0, jc = 0;
      uint32_t phase = 0;
      long long seq = 0;
      bool ok = true;
      for (long long gi = blockIdx.x; ok && gi < B.total_items; gi += gridDim.x) {
        while (jc + 1 < B.njobs && gi >= B.job[jc + 1].item0) ++jc;   // items ascend: the cursor only moves on
        const WtJob &J = B.job[jc];
        int m, tl, g, nci, p, q, r;
        wt_decode(J, gi - J.item0, m, tl, g, nci);
        wt_occ(J, tl, g, p, q, r);
        const int nkb = J.g.hv + J.g.ho;                       // 2 (hv + ho) halves, two per K block
        const uint32_t ahb = (uint32_t)S * A_HALF, bhb = (uint32_t)S * J.g.nc * 16;
        for (int kc = 0; kc < nkb; ++kc, ++seq) {
          const bool mine = rr == pw;
          if (++rr == B.nprod) rr = 0;
          if (mine) {
            int got = 1;
            if (lane == 0) {
              got = mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, B.err, ERR_TIMEOUT_EMPTY) ? 1 : 0;
              if (got) {
                last_seq[pw][stage] = seq;
                mbar_expect_tx(&full_bar[stage], 2 * (ahb + bhb));
              }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) { ok = false; break; }
            // The block's two K halves land S slices apart: [A h0][A h1][B h0][B h1].
            // Halves of one segment are consecutive in its image (one copy per
            // operand); a block across a segment boundary takes two.
            if (lane < 4) {
              const unsigned char *a0, *b0, *a1, *b1;
              int s0, s1;
              wt_src<S>(J, m, nci, p, q, r, 2 * kc, s0, a0, b0);
              wt_src<S>(J, m, nci, p, q, r, 2 * kc + 1, s1, a1, b1);
              unsigned char *sA = sm + (size_t)stage * B.slot, *sB = sA + 2 * ahb;
              const bool one = s0 == s1;
              if (lane == 0)      bulk_load(sA, a0, one ? 2 * ahb : ahb, &full_bar[stage]);
              else if (lane == 1) bulk_load(sB, b0, one ? 2 * bhb : bhb, &full_bar[stage]);
              else if (!one && lane == 2) bulk_load(sA + ahb, a1, ahb, &full_bar[stage]);
              else if (!one && lane == 3) bulk_load(sB + bhb, b1, bhb, &full_bar[stage]);
            }
            __syncwarp();
          }
          if (++stage == B.stages) { stage = 0; phase ^= 1u; }
        }
      }
    }
    // Before the CTA may exit, every issued copy has landed (bounded wait).  A
    // later copy into a stage is issued only after the previous one was
    // consumed, so only the latest copy into each stage can still be in flight.
    prod_bar();
    if (pw == 0 && lane == 0) {
      for (int s = 0; s < B.stages; ++s) {
        long long last = -1;
        for (int q = 0; q < NPROD; ++q) last = max(last, last_seq[q][s]);
        if (last < 0) continue;
        const uint32_t par = (uint32_t)((last / B.stages) & 1);
        const uint32_t a = smem_u32(&full_bar[s]);
        for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, par); ++it) {
          if ((it & 255) == 255) __nanosleep(128);
          if (it == WAIT_LIMIT - 1) atomicCAS(B.err, 0, ERR_TIMEOUT_TEARDOWN);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0, jc = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      for (long long gi = blockIdx.x; ok && gi < B.total_items; gi += gridDim.x) {
        while (jc + 1 < B.njobs && gi >= B.job[jc + 1].item0) ++jc;
        const WtJob &J = B.job[jc];
        const int nc = J.g.nc;
        const int nkb = J.g.hv + J.g.ho;
        const int nchain = (nkb + KCHAIN - 1) / KCHAIN;
        const uint32_t id = idesc(128, nc);
        const uint32_t ahb = (uint32_t)S * A_HALF, bhb = (uint32_t)S * nc * 16;
        for (int ch = 0; ok && ch < nchain; ++ch) {
          const int kc0 = ch * nkb / nchain, kc1 = (ch + 1) * nkb / nchain;
          // A new item needs both accumulators back from the drain.  A later
          // chain needs only L0, which the drain is still reading: its first
          // ndef K blocks issue their L1 products first, and their level-0
          // products (in K order, the first one restarting L0) follow once L0
          // is free, so the tensor pipe keeps working meanwhile.
          if (ch == 0) {
            if (!mbar_wait(&accempty_bar, aphase ^ 1u, &abort_flag, B.err, ERR_TIMEOUT_ACCEMPTY)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          }
          const int ndef = ch > 0 ? min(DEFER, kc1 - kc0) : 0;
          int dstage[DEFER];
          for (int kc = kc0; kc < kc1; ++kc) {
            if (!mbar_wait(&full_bar[stage], phase, &abort_flag, B.err, ERR_TIMEOUT_FULL)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sA = smem_u32(sm + (size_t)stage * B.slot);
            const uint32_t sB = sA + 2 * ahb;
            int n = 0;
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
              for (int b = 0; b < S - a; ++b) {
                if (a + b == 0) continue;                                          // levels >= 1 -> L1
                mma_bf16(tbase + (uint32_t)nc, sdesc(sA + a * A_HALF, ahb), sdesc(sB + b * nc * 16, bhb), id,
                         (kc == 0 && n == 0) ? 0u : 1u);
                ++n;
              }
            if (kc - kc0 < ndef) {
              dstage[kc - kc0] = stage;                                            // level 0 deferred
              if (++stage == B.stages) { stage = 0; phase ^= 1u; }
              if (kc - kc0 + 1 < ndef) continue;
              if (!mbar_wait(&accempty_bar, aphase ^ 1u, &abort_flag, B.err, ERR_TIMEOUT_ACCEMPTY)) { ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              for (int d = 0; d < ndef; ++d) {
                const uint32_t dA = smem_u32(sm + (size_t)dstage[d] * B.slot), dB = dA + 2 * ahb;
                mma_bf16(tbase, sdesc(dA, ahb), sdesc(dB, bhb), id, d > 0 ? 1u : 0u);   // level 0 -> L0
                mma_commit(&empty_bar[dstage[d]]);
              }
              continue;
            }
            mma_bf16(tbase, sdesc(sA, ahb), sdesc(sB, bhb), id, kc > kc0 ? 1u : 0u);  // level 0 -> L0
            mma_commit(&empty_bar[stage]);
            if (++stage == B.stages) { stage = 0; phase ^= 1u; }
          }
          if (!ok) break;
          mma_commit(&accfull_bar);
          aphase ^= 1u;
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(&teardown_bar);
      const uint32_t a = smem_u32(&teardown_bar);
      for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, 0); ++it) {
        if ((it & 255) == 255) __nanosleep(128);
        if (it == WAIT_LIMIT - 1) atomicCAS(B.err, 0, ERR_TIMEOUT_TEARDOWN);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain: TMEM -> row sums in registers -> Y
    const int et = tid - 64;                        // 0 .. 255
    const int quarter = warp & 3;                   // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;               // which half of the 16-column groups
    const int lrow = 32 * quarter + lane;           // row of the M tile
    const uint32_t trow = tbase + ((uint32_t)(32 * quarter) << 16);
    uint32_t aphase = 0;
    bool ok = true;
    bool dep_done = false;                          // the preceding launch has completed (see below)
    int jc = 0;
    for (long long gi = blockIdx.x; ok && gi < B.total_items; gi += gridDim.x) {
      while (jc + 1 < B.njobs && gi >= B.job[jc + 1].item0) ++jc;
      const WtJob &J = B.job[jc];
      const int nc = J.g.nc;
      const int nkb = J.g.hv + J.g.ho;
      const int nchain = (nkb + KCHAIN - 1) / KCHAIN;
      const int ng = nc / 16, gsplit = (ng + 1) / 2;
      const int g0 = half ? gsplit : 0, my = half ? ng - gsplit : gsplit;
      float v[MG][16];                                // this thread's row: running sum over chains
      for (int ch = 0; ch < nchain; ++ch) {
        if (et == 0) drain_ok = mbar_wait(&accfull_bar, aphase, &abort_flag, B.err, ERR_TIMEOUT_ACCFULL) ? 1 : 0;
        drain_bar();
        if (!drain_ok) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // The row's running sum lives in v: the first chain's L0 is read into
        // it, later chains add theirs (and the last chain L1 as well) one
        // 16-column group at a time; then the accumulators go back to the MMA
        // warp.
        const bool last = ch + 1 == nchain;
        if (ch == 0 && !last) {
#pragma unroll
          for (int gi2 = 0; gi2 < MG; ++gi2)
            if (gi2 < my) tmem_ld16(trow + (uint32_t)((g0 + gi2) * 16), v[gi2]);
          tmem_wait_ld();
        } else if constexpr (MG <= 7) {
#pragma unroll
          for (int gi2 = 0; gi2 < MG; ++gi2) {
            if (gi2 >= my) break;
            float l0[16], l1[16];
            tmem_ld16(trow + (uint32_t)((g0 + gi2) * 16), l0);
            if (last) tmem_ld16(trow + (uint32_t)(nc + (g0 + gi2) * 16), l1);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float x = last ? l0[e] + l1[e] : l0[e];
              v[gi2][e] = ch > 0 ? x + v[gi2][e] : x;
            }
          }
        } else {
          // the same sums, eight columns at a time: with 8 groups of 16 in v,
          // 16-column temporaries would spill
#pragma unroll
          for (int gi2 = 0; gi2 < MG; ++gi2) {
            if (gi2 >= my) break;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              float l0[8], l1[8];
              tmem_ld8(trow + (uint32_t)((g0 + gi2) * 16 + 8 * hh), l0);
              if (last) tmem_ld8(trow + (uint32_t)(nc + (g0 + gi2) * 16 + 8 * hh), l1);
              tmem_wait_ld();
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const float x = last ? l0[e] + l1[e] : l0[e];
                v[gi2][8 * hh + e] = ch > 0 ? x + v[gi2][8 * hh + e] : x;
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        drain_bar();
        if (et == 0) mbar_arrive(&accempty_bar);
        aphase ^= 1u;
        if (!last) continue;
        // The last chain: the row goes into the job's W buffer Y[triplet][a][b][c].
        // F(i,j,k) stores its row (a, b): the four lanes of a quad first trade
        // 16-byte chunks (a 4 x 4 transpose in two xor shuffles) so that every
        // warp store covers 64 contiguous bytes of each of 8 rows.  F(i,k,j)
        // (row (a, c)) and F(j,k,i) (row (b, c)) add theirs column by column
        // with reductions in L2 (not read back, so nothing waits on them); the
        // warp's 32 lanes hold 32 consecutive c, so each column's reductions
        // cover 128 contiguous bytes.  Each W element has one writer per launch
        // and the launches are ordered, so every element is the same IEEE sum
        // on every run.
        int m, tl, g, nci;
        wt_decode(J, gi - J.item0, m, tl, g, nci);
        const int vo = J.g.v, vc = J.g.vc;
        const int row = m * MROWS + lrow;
        // Y is written by the preceding F launch (or read by the preceding
        // energy launch): under a programmatic launch, everything before
        // this point overlapped that launch's tail
        if (!dep_done) { asm volatile("griddepcontrol.wait;" ::: "memory"); dep_done = true; }
        const int zb = nci * nc + g0 * 16;              // first column this thread holds
        float *Wf = J.y + (size_t)tl * vo * vo * vc;
        if (g == 0) {
          const int q = lane & 3;                       // place in the quad
          const int r0 = row - q;                       // the quad's first row
#pragma unroll
          for (int gi2 = 0; gi2 < MG; ++gi2) {
            if (gi2 >= my) break;                       // warp-uniform
            float4 X[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
              X[k] = make_float4(v[gi2][4 * k], v[gi2][4 * k + 1], v[gi2][4 * k + 2], v[gi2][4 * k + 3]);
            // lane q held chunk k of row r0 + q; afterwards X[r] = chunk q of row r0 + r
#pragma unroll
            for (int b = 2; b >= 1; b >>= 1) {
              const bool up = (q & b) != 0;
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                if (k & b) continue;
                const float4 snd = up ? X[k] : X[k | b];
                float4 rcv;
                rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, b);
                rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, b);
                rcv.z = __shfl_xor_sync(0xffffffffu, snd.z, b);
                rcv.w = __shfl_xor_sync(0xffffffffu, snd.w, b);
                if (up) X[k] = rcv;
                else X[k | b] = rcv;
              }
            }
            const int col = zb + gi2 * 16 + 4 * q;
#pragma unroll
            for (int r = 0; r < 4; ++r)
              if (r0 + r < vo * vo && col < vo) *(float4 *)(Wf + (size_t)(r0 + r) * vc + col) = X[r];
          }
        } else {
          if (row >= vo * vo) continue;
          const int p = row / vo, c = row - p * vo;
          const size_t st = (g == 1) ? (size_t)vc : (size_t)vo * vc;
          float *dst = Wf + ((g == 1) ? (size_t)p * vo * vc : (size_t)p * vc) + c + (size_t)zb * st;
#pragma unroll
          for (int gi2 = 0; gi2 < MG; ++gi2) {
            if (gi2 >= my) break;
#pragma unroll
            for (int e = 0; e < 16; ++e)
              if (zb + gi2 * 16 + e < vo) atomicAdd(dst + (size_t)(gi2 * 16 + e) * st, v[gi2][e]);
          }
        }
      }
      if (!ok) break;
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512));
  }
}

// ---------------------------------------------------------------- energy kernel
//
// One CTA per SM walks its items (triplet, chunk of consecutive orbits).  The
// producer warp owns the walk: per orbit it fills one of two "V sets" (the
// eighteen 16 x 16 G tiles and nine 16-entry t1 rows the orbit's V needs, by
// TMA, plus a small record of the orbit: triplet, tiles, distinct blocks,
// item) and then loads the orbit's distinct W blocks (one 16^3 box of the
// triplet's W buffer each, 4-D tensor map, zero-filled where an index reaches
// v) into a ring of staging slots.  The consumer warps copy each box into its
// padded W block, release the slot warp by warp, evaluate the orbit's energy
// once its blocks are in place and release the V set; so the next orbit's
// loads fly while the current orbit's energy is evaluated, and the consumers
// meet at a CTA barrier only twice per orbit.
//
// G tiles: G_pq^uw = (p u|q w) for the occupied pairs (p, q) = (j, k), (i, k),
// (i, j) and the six ordered pairs (u, w) of the orbit's tile positions.  The
// FP32 copy of ovov holds (p u|q w) in both orders, [p][u][q][w] and
// [q][w][p][u], so each tile lands in the orientation whose reads in the
// energy loop are free of bank conflicts: [u][w] for (a,b), (a,c), (c,a),
// (c,b) and [w][u] for (b,a), (b,c).

// Index of the ordered pair (u, w) of distinct tile positions:
// (0,1) (1,0) (0,2) (2,0) (1,2) (2,1)
__host__ __device__ constexpr int tpair(int u, int w) {
  return (u == 0) ? (w == 1 ? 0 : 2) : (u == 1) ? (w == 0 ? 1 : 4) : (w == 0 ? 3 : 5);
}
__host__ __device__ constexpr int tpair_u(int tp) { return tp == 0 || tp == 2 ? 0 : (tp == 1 || tp == 4 ? 1 : 2); }
__host__ __device__ constexpr int tpair_w(int tp) { return tp == 1 || tp == 3 ? 0 : (tp == 0 || tp == 5 ? 1 : 2); }
__host__ __device__ constexpr bool tpair_swapped(int tp) { return tp == 1 || tp == 4; }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3}], [%4];"
               :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
  asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3, %4, %5}], [%6];"
               :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t *bar) {
  asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
               " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
               :: "r"(smem_u32(dst)), "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
               : "memory");
}

// What the consumers need to know about the orbit of a V set.
struct OrbMeta {
  long long pidx;      // partial slot of the orbit's item
  float eh, el;        // e_i + e_j + e_k as a float pair (hi + lo)
  int jc, tl;          // job and triplet in the job's block
  int tl3[3];          // tiles P >= Q >= R
  int blk[6];          // distinct block of each formal permutation (orbit_blocks)
  int last;            // last orbit of its item
  int valid;           // 0: no more orbits
};

// Float pair arithmetic: h + l carries about 48 significant bits (Knuth's
// TwoSum for additions, Dekker's products with an FMA).
__device__ __forceinline__ void ff_add2(float &h, float &l, float h2, float l2) {
  const float s = h + h2, bp = s - h;
  l += ((h - (s - bp)) + (h2 - bp)) + l2;
  h = s;
}
// Renormalise a pair so that |l| <= ulp(h) / 2 (Dekker's fast TwoSum; |h| >= |l|).
__device__ __forceinline__ void ff_norm(float &h, float &l) {
  const float s = h + l;
  l -= s - h;
  h = s;
}
// Reciprocal of the pair (h, l) as a pair: r = fl(1/h) corrected by one Newton
// step on the exact residual 1 - (h + l) r, formed with FMAs.
__device__ __forceinline__ void ff_rcp(float h, float l, float &rh, float &rl) {
  rh = __frcp_rn(h);
  float e = fmaf(-h, rh, 1.f);
  e = fmaf(-l, rh, e);
  rl = rh * e;
}
// (h, l) * x as a pair for a float x (Dekker's product with an FMA).
__device__ __forceinline__ void ff_mulf(float h, float l, float x, float &ph, float &pl) {
  ph = h * x;
  pl = fmaf(h, x, -ph) + l * x;
}
// (h, l) / 6 as a pair: times the pair of 1/6.
__device__ __forceinline__ void ff_mul_sixth(float &h, float &l) {
  constexpr float c_h = 1.f / 6.f;
  constexpr float c_l = (float)(1.0 / 6.0 - (double)(1.f / 6.f));
  const float ph = h * c_h;
  l = fmaf(h, c_h, -ph) + (h * c_l + l * c_h);
  h = ph;
}

__device__ __forceinline__ void cons_bar() { asm volatile("bar.sync 1, %0;" :: "n"(EN_CONSUMERS) : "memory"); }

__global__ void __launch_bounds__(EN_THREADS, 1)
tc_energy_kernel(const __grid_constant__ EnBatch B) {
  extern __shared__ __align__(1024) unsigned char en_raw[];
  float *stg = (float *)(((uintptr_t)en_raw + 1023) & ~(uintptr_t)1023);   // W staging slots [EN_SLOTS][16^3]
  float *vset = stg + EN_SLOTS * BOXF;                                      // V sets [EN_VSETS][GSET_FLOATS]
  float *Wsm = vset + EN_VSETS * GSET_FLOATS;                               // padded W blocks [6][WBLK]
  __shared__ __align__(8) uint64_t full_bar[EN_SLOTS], empty_bar[EN_SLOTS], vfull_bar[EN_VSETS],
      vempty_bar[EN_VSETS];
  __shared__ OrbMeta meta[EN_VSETS];
  __shared__ float red[EN_WARPS][4];
  __shared__ volatile int en_abort;          // set by a wait that gave up
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int k = 0; k < EN_SLOTS; ++k) { mbar_init(&full_bar[k], 1); mbar_init(&empty_bar[k], EN_WARPS); }
    for (int k = 0; k < EN_VSETS; ++k) { mbar_init(&vfull_bar[k], 1); mbar_init(&vempty_bar[k], EN_WARPS); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    en_abort = 0;
  }
  __syncthreads();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

  if (warp == EN_WARPS) {
    // ------------------------------------------------ producer: the CTA's walk
    if (lane == 0) {
      int ws = 0, vs = 0;                  // next staging slot, next V set
      uint32_t wpar = 1, vpar = 1;         // parities of their "free" phases (fresh barriers count as free)
      long long nW = 0, nV = 0;            // loads issued
      bool ok = true;
      bool dep_done = false;               // the launch that wrote Y has completed
      int jc = 0;
      for (long long gi = blockIdx.x; ok && gi < B.total_items; gi += gridDim.x) {
        while (jc + 1 < B.njobs && gi >= B.job[jc + 1].item0) ++jc;
        const EnJob &J = B.job[jc];
        const Dims &d = J.d;
        const long long q = gi - J.item0;
        const int tl = (int)(q / d.items_per_trip), chunk = (int)(q % d.items_per_trip);
        const int ob0 = chunk * d.orb_per_item, ob1 = min(d.n_orb, ob0 + d.orb_per_item);
        const int4 og = J.orb[ob0];                  // the item's first orbit; the next ones follow
        int tl3[3] = {og.x, og.y, og.z};
        const int4 tr = J.trip[J.t0 + tl];
        const int occ[3] = {tr.x, tr.y, tr.z};
        const double e3 = J.eps[tr.x] + J.eps[tr.y] + J.eps[tr.z];
        const float eh = (float)e3, el = (float)(e3 - (double)eh);
        const long long pidx = (long long)(J.t0 + tl) * d.items_per_trip + chunk;
        for (int ob = ob0; ob < ob1; ++ob) {
          int blk[6];
          orbit_blocks(tl3, blk);
          // the orbit's V set and record
          if (!mbar_wait(&vempty_bar[vs], vpar, &en_abort, B.err, ERR_TIMEOUT_EMPTY)) { ok = false; break; }
          OrbMeta &m = meta[vs];
          m.pidx = pidx;
          m.eh = eh;
          m.el = el;
          m.jc = jc;
          m.tl = tl;
          for (int u = 0; u < 3; ++u) m.tl3[u] = tl3[u];
          for (int s = 0; s < 6; ++s) m.blk[s] = blk[s];
          m.last = ob + 1 == ob1;
          m.valid = 1;
          float *V = vset + (size_t)vs * GSET_FLOATS;
          mbar_expect_tx(&vfull_bar[vs], GSET_TX);
          for (int op = 0; op < 3; ++op) {
            const int p0 = op == 0 ? occ[1] : occ[0], q0 = op == 2 ? occ[1] : occ[2];
            for (int tp = 0; tp < 6; ++tp) {
              const int Ut = tl3[tpair_u(tp)] * NT, Wt = tl3[tpair_w(tp)] * NT;
              float *dst = V + (op * 6 + tp) * NT * NT;
              if (tpair_swapped(tp)) tma_load_5d(dst, &J.gmap, Ut, p0, Wt, q0, 1, &vfull_bar[vs]);
              else                   tma_load_5d(dst, &J.gmap, Wt, q0, Ut, p0, 0, &vfull_bar[vs]);
            }
            for (int pos = 0; pos < 3; ++pos)
              tma_load_2d(V + G_FLOATS + (op * 3 + pos) * T1_ROW, &J.tmap, tl3[pos] * NT, occ[op], &vfull_bar[vs]);
          }
          ++nV;
          if (++vs == EN_VSETS) { vs = 0; vpar ^= 1u; }
          // the orbit's distinct W blocks, in the order of their permutation index
          for (int s = 0; s < 6 && ok; ++s) {
            if (blk[s] != s) continue;
            if (!mbar_wait(&empty_bar[ws], wpar, &en_abort, B.err, ERR_TIMEOUT_EMPTY)) { ok = false; break; }
            // under a programmatic launch the V sets above may already be in
            // flight; Y needs the preceding W-term launch complete
            if (!dep_done) { asm volatile("griddepcontrol.wait;" ::: "memory"); dep_done = true; }
            mbar_expect_tx(&full_bar[ws], BOXF * 4);
            tma_load_4d(stg + (size_t)ws * BOXF, &J.ymap, tl3[perm3(s, 2)] * NT, tl3[perm3(s, 1)] * NT,
                        tl3[perm3(s, 0)] * NT, tl, &full_bar[ws]);
            ++nW;
            if (++ws == EN_SLOTS) { ws = 0; wpar ^= 1u; }
          }
          // the orbit table's order, P >= Q >= R lexicographic, as an odometer
          if (tl3[2] < tl3[1]) ++tl3[2];
          else if (tl3[1] < tl3[0]) { ++tl3[1]; tl3[2] = 0; }
          else { ++tl3[0]; tl3[1] = 0; tl3[2] = 0; }
        }
      }
      // end of the walk: a record with valid = 0 (its set's previous load has
      // been consumed once the set is free again)
      if (ok && mbar_wait(&vempty_bar[vs], vpar, &en_abort, B.err, ERR_TIMEOUT_EMPTY)) {
        meta[vs].valid = 0;
        for (int s = 0; s < 6; ++s) meta[vs].blk[s] = -1;
        mbar_arrive(&vfull_bar[vs]);
      }
      // loads still in flight land before the CTA may exit (bounded): the
      // latest load into each staging slot and into each V set (after an end
      // record, not the one into the end record's set, which was free)
      for (long long k = (nW > EN_SLOTS ? nW - EN_SLOTS : 0); k < nW; ++k) {
        const uint32_t a = smem_u32(&full_bar[k % EN_SLOTS]);
        for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, (uint32_t)((k / EN_SLOTS) & 1)); ++it)
          if ((it & 255) == 255) __nanosleep(128);
      }
      const long long vfly = ok ? EN_VSETS - 1 : EN_VSETS;
      for (long long k = (nV > vfly ? nV - vfly : 0); k < nV; ++k) {
        const uint32_t a = smem_u32(&vfull_bar[k % EN_VSETS]);
        for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, (uint32_t)((k / EN_VSETS) & 1)); ++it)
          if ((it & 255) == 255) __nanosleep(128);
      }
    }
    __syncwarp();
    __syncthreads();
    return;
  }

  // -------------------------------------------------- consumers
  // Thread (pr, hf) takes the point row (la, lb) = (pr / 16, pr % 16) of an
  // orbit and half hf of its c range.  The W and V parts of E_(T) (E[4] and
  // E[5]_ST) run as float pairs over the item's orbits.
  const int pr = tid & (NT * NT - 1), hf = tid >> 8;
  const int la = pr >> 4, lb = pr & 15;
  float a4h = 0.f, a4l = 0.f, a5h = 0.f, a5l = 0.f;
  int ws = 0, vs = 0;
  uint32_t wpar = 0, vpar = 0;
  while (true) {
    mbar_wait(&vfull_bar[vs], vpar, &en_abort, B.err, ERR_TIMEOUT_FULL);
    const OrbMeta &m = meta[vs];
    const int valid = m.valid, jc = m.jc, last = m.last;
    const int T0 = m.tl3[0], T1 = m.tl3[1], T2 = m.tl3[2];
    int blk[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) blk[s] = m.blk[s];
    // the orbit's W blocks into their padded form
#pragma unroll 1
    for (int s = 0; s < 6; ++s) {
      if (blk[s] != s) continue;
      mbar_wait(&full_bar[ws], wpar, &en_abort, B.err, ERR_TIMEOUT_FULL);
      const float4 *sb = (const float4 *)(stg + (size_t)ws * BOXF);
      float *Wb = Wsm + s * WBLK;
#pragma unroll
      for (int k = 0; k < BOXF / 4 / EN_CONSUMERS; ++k) {
        const int e4 = tid + k * EN_CONSUMERS;            // float4 index: (x, y, z4)
        const float4 a0 = sb[e4];
        float *w = Wb + (e4 >> 6) * WX + ((e4 >> 2) & 15) * WY + (e4 & 3) * 4;
        w[0] = a0.x;
        w[1] = a0.y;
        w[2] = a0.z;
        w[3] = a0.w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty_bar[ws]);      // this warp is done with the slot
      if (++ws == EN_SLOTS) { ws = 0; wpar ^= 1u; }
    }
    cons_bar();                                        // W blocks in place; a failed wait shows here
    if (en_abort || !valid) break;
    const EnJob &J = B.job[jc];
    const int o = J.d.o, v = J.d.v;
    const float *V = vset + (size_t)vs * GSET_FLOATS;
    const float *G = V, *t1s = V + G_FLOATS;
    const int ga = T0 * NT + la, gb = T1 * NT + lb;
    if (ga < v && gb < v && ga >= gb) {
      // D = e_i + e_j + e_k - e_a - e_b - e_c as a float pair (about 48
      // significant bits): the row's part here, e_c per point below
      const int ne = o + v;
      float dh = m.eh, dl = m.el;
      ff_add2(dh, dl, -__ldg(J.epsf + o + ga), -__ldg(J.epsf + ne + o + ga));
      ff_add2(dh, dl, -__ldg(J.epsf + o + gb), -__ldg(J.epsf + ne + o + gb));
      ff_norm(dh, dl);
      // V inputs of the row that do not depend on c: t1 at the a and b
      // positions, G at the position pairs (a, b) and (b, a); op 0, 1, 2 =
      // occupied pair (j, k), (i, k), (i, j) for G and i, j, k for t1
      float ta[3], tb[3], gab[3], gba[3];
#pragma unroll
      for (int op = 0; op < 3; ++op) {
        ta[op] = t1s[(op * 3 + 0) * T1_ROW + la];
        tb[op] = t1s[(op * 3 + 1) * T1_ROW + lb];
        gab[op] = G[(op * 6 + tpair(0, 1)) * NT * NT + la * NT + lb];          // [a][b]
        gba[op] = G[(op * 6 + tpair(1, 0)) * NT * NT + la * NT + lb];          // [a][b] (swapped tile)
      }
      // This thread's 8 points (la, lb, lc0 + u): every shared read below is a
      // row base plus a compile-time offset in u.
      const int lc0 = hf * 8;
      const float *tcp = t1s + 2 * T1_ROW + lc0;                        // t1 at the c position
      const float *gacp = G + tpair(0, 2) * NT * NT + la * NT + lc0;   // [a][c]
      const float *gcap = G + tpair(2, 0) * NT * NT + lc0 * NT + la;   // [c][a]
      const float *gbcp = G + tpair(1, 2) * NT * NT + lc0 * NT + lb;   // [c][b] (swapped tile)
      const float *gcbp = G + tpair(2, 1) * NT * NT + lc0 * NT + lb;   // [c][b]
      // W at permutation s of the point: block blk[s], index l3[p0] WX + l3[p1] WY + l3[p2]
      auto wcoef = [](int s, int pos) { return perm3(s, 0) == pos ? WX : (perm3(s, 1) == pos ? WY : 1); };
      int wo[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) wo[s] = blk[s] * WBLK + la * wcoef(s, 0) + lb * wcoef(s, 1) + lc0 * wcoef(s, 2);
      const float *ecp = J.epsf + o + T2 * NT + lc0;
      float r4h = 0.f, r4l = 0.f, r5h = 0.f, r5l = 0.f;   // the row's sums (float pairs)
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int gc = T2 * NT + lc0 + u;
        if (gc >= v || gb < gc) continue;
        float tcc[3], gac[3], gca[3], gbc[3], gcb[3];
#pragma unroll
        for (int op = 0; op < 3; ++op) {
          tcc[op] = tcp[op * 3 * T1_ROW + u];
          gac[op] = gacp[op * 6 * NT * NT + u];
          gca[op] = gcap[op * 6 * NT * NT + u * NT];
          gbc[op] = gbcp[op * 6 * NT * NT + u * NT];
          gcb[op] = gcbp[op * 6 * NT * NT + u * NT];
        }
        // t1 of op at position pos, G of op at positions (pu, pw)
        auto tv = [&](int op, int pos) { return pos == 0 ? ta[op] : (pos == 1 ? tb[op] : tcc[op]); };
        auto gv = [&](int op, int pu, int pw) {
          return pu == 0 ? (pw == 1 ? gab[op] : gac[op])
               : pu == 1 ? (pw == 0 ? gba[op] : gbc[op])
                         : (pw == 0 ? gca[op] : gcb[op]);
        };
        float wv[6], vv[6];
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          const int p0 = perm3(s, 0), p1 = perm3(s, 1), p2 = perm3(s, 2);
          wv[s] = Wsm[wo[s] + u * wcoef(s, 2)];
          // V (Eq. 3) at (x, y, z) = positions (p0, p1, p2) of the point:
          // t_i^x G_jk^yz + t_j^y G_ik^xz + t_k^z G_ij^xy
          vv[s] = tv(0, p0) * gv(0, p1, p2) + tv(1, p1) * gv(1, p0, p2) + tv(2, p2) * gv(2, p0, p1);
        }
        // The Eq. 1 bracket at permutation s is 3 w_s + (se - 2 so) for even s
        // and 3 w_s + (so - 2 se) for odd s (se, so: sums of w over the even and
        // odd permutations), so
        //   sum_s w_s br_s = 3 sum_s w_s^2 + se^2 + so^2 - 4 se so,
        //   sum_s v_s br_s = 3 sum_s v_s w_s + ve (se - 2 so) + vo (so - 2 se).
        const float se = wv[0] + wv[3] + wv[4], so = wv[1] + wv[2] + wv[5];
        const float ve = vv[0] + vv[3] + vv[4], vo = vv[1] + vv[2] + vv[5];
        float ww = wv[0] * wv[0], vw = vv[0] * wv[0];
#pragma unroll
        for (int s = 1; s < 6; ++s) {
          ww = fmaf(wv[s], wv[s], ww);
          vw = fmaf(vv[s], wv[s], vw);
        }
        const float sumf4 = fmaf(3.f, ww, fmaf(se, se - 4.f * so, so * so));
        const float sumf5 = fmaf(3.f, vw, fmaf(ve, se - 2.f * so, vo * (so - 2.f * se)));
        // 1/D as a float pair (rh, rl), scaled by the point's share of the
        // bracket sum: 1 for distinct a > b > c, 1/2 with two equal, 1/6 for a = b = c
        float Dh = dh, Dl = dl;
        ff_add2(Dh, Dl, -__ldg(ecp + u), -__ldg(ecp + ne + u));
        ff_norm(Dh, Dl);
        float rh, rl;
        ff_rcp(Dh, Dl, rh, rl);
        if (ga == gc) ff_mul_sixth(rh, rl);
        else if (ga == gb || gb == gc) { rh *= 0.5f; rl *= 0.5f; }
        // the point's two quotients as float pairs, added to the row's pairs
        float qh, ql;
        ff_mulf(rh, rl, sumf4, qh, ql);
        ff_add2(r4h, r4l, qh, ql);
        ff_mulf(rh, rl, sumf5, qh, ql);
        ff_add2(r5h, r5l, qh, ql);
      }
      ff_add2(a4h, a4l, r4h, r4l);
      ff_add2(a5h, a5l, r5h, r5l);
    }
    const long long pidx = m.pidx;
    __syncwarp();
    if (lane == 0) mbar_arrive(&vempty_bar[vs]);       // this warp is done with the V set
    if (++vs == EN_VSETS) { vs = 0; vpar ^= 1u; }
    if (last) {
      // the item's partial: fixed-order reduction of the float pairs (warps,
      // then the 16 warp sums by warp 0), written in FP64
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float h4 = __shfl_down_sync(0xffffffffu, a4h, off), l4 = __shfl_down_sync(0xffffffffu, a4l, off);
        const float h5 = __shfl_down_sync(0xffffffffu, a5h, off), l5 = __shfl_down_sync(0xffffffffu, a5l, off);
        ff_add2(a4h, a4l, h4, l4);
        ff_add2(a5h, a5l, h5, l5);
      }
      if (lane == 0) { red[warp][0] = a4h; red[warp][1] = a4l; red[warp][2] = a5h; red[warp][3] = a5l; }
      cons_bar();                                      // also: Wsm reads done before the next orbit's copies
      if (warp == 0) {
        a4h = lane < EN_WARPS ? red[lane][0] : 0.f;
        a4l = lane < EN_WARPS ? red[lane][1] : 0.f;
        a5h = lane < EN_WARPS ? red[lane][2] : 0.f;
        a5l = lane < EN_WARPS ? red[lane][3] : 0.f;
#pragma unroll
        for (int off = EN_WARPS / 2; off > 0; off >>= 1) {
          const float h4 = __shfl_down_sync(0xffffffffu, a4h, off), l4 = __shfl_down_sync(0xffffffffu, a4l, off);
          const float h5 = __shfl_down_sync(0xffffffffu, a5h, off), l5 = __shfl_down_sync(0xffffffffu, a5l, off);
          ff_add2(a4h, a4l, h4, l4);
          ff_add2(a5h, a5l, h5, l5);
        }
        if (lane == 0) {
          const double e4 = (double)a4h + (double)a4l, e5 = (double)a5h + (double)a5l;
          J.partial[2 * pidx] = e4 + e5;
          J.partial[2 * pidx + 1] = e5;
        }
      }
      a4h = a4l = a5h = a5l = 0.f;
    } else {
      cons_bar();                                      // Wsm reads done before the next orbit's copies
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- operand images

// One thread per (K half, row): reads 8 consecutive K values of one operand
// row, splits them into S BF16 slices and writes 16 bytes per slice at the
// row's place in the no-swizzle K-major half (core matrices of 8 rows x 16
// bytes, 8-row groups 128 bytes apart).  An image is a sequence of halves,
// each S slices of rows x 16 bytes; rows or K values outside the tensors are
// zero.
//   kind 0  A  [p][m][hv]        row (x, y), K f:  (p x | y f)            = ovvv[p][x][y][f]
//   kind 1  A  [p][m][hv]        row (x, y), K f:  (p y | x f)            = ovvv[p][y][x][f]
//   kind 2  A  [p][m][ho]        row (x, y), K l:  t_lp^xy = t_pl^yx      = t2[p][l][y][x]
//   kind 3  A  [p][m][ho]        row (x, y), K l:  t_lp^yx = t_pl^xy      = t2[p][l][x][y]
//   kind 4  B  [r][q][nc][hv]    row z,      K f:  t_rq^zf                = t2[r][q][z][f]
//   kind 5  B  [r][q][nc][ho]    row z,      K l:  -(r z | q l)           = -ovoo[r][z][q][l]
// (kinds 2 and 3 read t_lp^.. as t_pl^.. with the virtual pair swapped, which
// keeps the reads coalesced).  Every kind's halves are ordered by the first
// occupied index of the tensor they read (p, or r), so the threads of one
// first-index range are the contiguous range [e_begin, e_end) of the image's
// (half, row) index.
__global__ void build_image(int kind, const double *__restrict__ src, SplitGeom G, long long e_begin,
                            long long e_end, unsigned char *__restrict__ out) {
  const int o = G.o, v = G.v, S = G.S;
  const bool isA = kind < 4;
  const int rows = isA ? MROWS : G.nc;
  const int nh = (kind == 0 || kind == 1 || kind == 4) ? G.hv : G.ho;
  const int kmax = (kind == 0 || kind == 1 || kind == 4) ? v : o;
  const long long nhalf = isA ? (long long)o * G.mt * nh : (long long)o * o * G.nch * nh;
  const size_t half_bytes = (size_t)rows * 16;
  const long long total = min(nhalf * rows, e_end);
  const long long vv = (long long)v * v;
  for (long long e = e_begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows);
    const long long hb = e / rows;
    const int h = (int)(hb % nh);
    const long long rest = hb / nh;
    const int k0 = h * 8;
    double x[8];
    if (isA) {
      const int m = (int)(rest % G.mt);
      const long long p = rest / G.mt;
      const long long row = (long long)m * MROWS + r;
      const bool valid = row < vv;
      const long long xi = valid ? row / v : 0, yi = valid ? row % v : 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u;
        double val = 0.0;
        if (valid && k < kmax) {
          if (kind == 0)      val = src[((p * v + xi) * v + yi) * v + k];
          else if (kind == 1) val = src[((p * v + yi) * v + xi) * v + k];
          else if (kind == 2) val = src[((p * o + k) * v + yi) * v + xi];
          else                val = src[((p * o + k) * v + xi) * v + yi];
        }
        x[u] = val;
      }
    } else {
      const int nci = (int)(rest % G.nch);
      const long long pair = rest / G.nch;               // r * o + q
      const long long rr = pair / o, qq = pair % o;
      const int z = nci * G.nc + r;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u;
        double val = 0.0;
        if (z < v && k < kmax) {
          if (kind == 4) val = src[((rr * o + qq) * v + z) * v + k];
          else           val = -src[((rr * v + z) * o + qq) * o + k];
        }
        x[u] = val;
      }
    }
    // position of row r in its half: 8-row group r/8, row r%8
    const int off = (r >> 3) * 128 + (r & 7) * 16;
    unsigned char *base = out + (size_t)hb * S * half_bytes + off;
    for (int p = 0; p < S; ++p) {
      __align__(16) __nv_bfloat16 b16[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        b16[u] = __double2bfloat16(x[u]);
        x[u] -= (double)__bfloat162float(b16[u]);        // exact FP64 residual
      }
      *(uint4 *)(base + (size_t)p * half_bytes) = *(const uint4 *)b16;
    }
  }
}

// FP32 copy of a [rows][cols] array with rows ld floats apart (zero beyond cols).
__global__ void f32_rows(const double *__restrict__ in, long long rows, int cols, int ld, float *__restrict__ out) {
  const long long n = rows * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / ld;
    const int c = (int)(e - r * ld);
    out[e] = c < cols ? (float)in[r * cols + c] : 0.f;
  }
}

// Float pair of each value: out[e] = fl(x), out[n + e] = fl(x - fl(x)).
__global__ void f32_hilo(const double *__restrict__ in, int n, float *__restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float h = (float)in[e];
    out[e] = h;
    out[n + e] = (float)(in[e] - (double)h);
  }
}

// FP32 (p u|q w) in both orders, rows vc floats long (zero beyond v):
// out[0][p][u][q][w] = ovov[p][u][q][w], out[1][q][w][p][u] = ovov[p][u][q][w],
// for the entries read from ovov rows p in [p0, p1) (ovov's first index: the
// first index of out[0], the third of out[1]).
__global__ void ovov_f32(const double *__restrict__ ovov, int o, int v, int vc, int p0, int p1,
                         float *__restrict__ out) {
  const int np = p1 - p0;
  const long long half = (long long)o * v * o * vc, part = (long long)np * v * o * vc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 2 * part;
       e += (long long)gridDim.x * blockDim.x) {
    const int h = e >= part;
    long long r = e - h * part;
    const int x3 = (int)(r % vc);
    r /= vc;
    int x0, x1, x2;
    if (h == 0) {
      x2 = (int)(r % o);
      r /= o;
      x1 = (int)(r % v);
      x0 = p0 + (int)(r / v);
    } else {
      x2 = p0 + (int)(r % np);
      r /= np;
      x1 = (int)(r % v);
      x0 = (int)(r / v);
    }
    float val = 0.f;
    if (x3 < v)
      val = (float)(h == 0 ? ovov[(((long long)x0 * v + x1) * o + x2) * v + x3]
                           : ovov[(((long long)x2 * v + x3) * o + x0) * v + x1]);
    out[h * half + (((long long)x0 * v + x1) * o + x2) * vc + x3] = val;
  }
}

// ---------------------------------------------------------------- host side

struct WtShape {
  int stages, nprod;
  size_t slot, smem;
};

// Shared-memory plan of a W-term launch whose widest N chunk is ncmax.
WtShape wt_shape(int S, int ncmax) {
  WtShape s{};
  s.slot = (size_t)S * A_BLK + (size_t)S * ncmax * 32;
  const long long st = ((long long)SMEM_DYN_MAX - 1024) / (long long)s.slot;
  s.stages = (int)std::min<long long>(MAX_STAGES, st);
  // The producers' parity waits on the empty barriers stay unambiguous only
  // while a producer is at most one ring cycle ahead of a stage's last use,
  // which the in-order MMA consumer guarantees when stages >= producers.
  s.nprod = std::min(NPROD, s.stages);
  s.smem = 1024 + (size_t)s.stages * s.slot;
  return s;
}

using WtKernel = void (*)(WtBatch);

// The W-term kernel instance for S slices and a widest N chunk of ncmax columns.
WtKernel wt_kernel(int S, int ncmax) {
  const bool wide = ncmax > NC_NARROW;
  switch (S) {
    case 2: return wide ? tc_wterm_kernel<2, 8> : tc_wterm_kernel<2, 7>;
    case 3: return wide ? tc_wterm_kernel<3, 8> : tc_wterm_kernel<3, 7>;
    default: return tc_wterm_kernel<4, 7>;
  }
}

void wt_params(WtKernel fn, const WtBatch &b, int grid, size_t smem, void **args, cudaKernelNodeParams *p) {
  args[0] = (void *)&b;
  *p = cudaKernelNodeParams{};
  p->func = (void *)fn;
  p->gridDim = dim3(grid);
  p->blockDim = dim3(THREADS);
  p->sharedMemBytes = (unsigned)smem;
  p->kernelParams = args;
}

// Item offsets, shared-memory plan, grids and W-term kernel instance of a
// W-term batch and an energy batch; sets the kernels' shared-memory limits.
cudaError_t prepare(WtBatch &wb, EnBatch &eb, int S, int num_sms, int *wgrid, int *egrid, size_t *wsmem,
                    WtKernel *wfn) {
  if (S < 2 || S > MAXS || wb.njobs < 1 || wb.njobs > MAX_BATCH || eb.njobs != wb.njobs) return cudaErrorInvalidValue;
  long long total = 0;
  int ncmax = 16;
  for (int j = 0; j < wb.njobs; ++j) {
    WtJob &J = wb.job[j];
    if (J.g.nc > (S >= 4 ? NCMAX_S4 : NCMAX) || J.g.S != S) return cudaErrorInvalidValue;
    J.item0 = total;
    total += (long long)J.g.mt * J.nt * J.g.nch;
    ncmax = std::max(ncmax, J.g.nc);
  }
  wb.total_items = total;
  const WtShape sh = wt_shape(S, ncmax);
  if (sh.stages <= DEFER) return cudaErrorInvalidValue;     // deferred K blocks hold stages
  wb.stages = sh.stages;
  wb.nprod = sh.nprod;
  wb.slot = sh.slot;
  *wsmem = sh.smem;
  long long etotal = 0;
  for (int j = 0; j < eb.njobs; ++j) {
    eb.job[j].item0 = etotal;
    etotal += (long long)eb.job[j].nt * eb.job[j].d.items_per_trip;
  }
  eb.total_items = etotal;
  *wgrid = (int)std::max<long long>(1, std::min<long long>(num_sms, total));
  *egrid = (int)std::max<long long>(1, std::min<long long>(num_sms, etotal));
  *wfn = wt_kernel(S, ncmax);
  cudaError_t e = cudaFuncSetAttribute(*wfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, EN_SMEM);
  return e;
}

}  // namespace

int split_tile() { return NT; }

int split_orb_per_item(int o, int v, int S) {
  const SplitGeom g = split_geom(o, v, S);
  const long long T = (v + NT - 1) / NT;
  const long long n_orb = T * (T + 1) * (T + 2) / 6;
  const long long opi = (long long)g.nb * n_orb / (8LL * 152);
  return (int)std::max<long long>(1, std::min<long long>(opi, n_orb));
}

SplitGeom split_geom(int o, int v, int S) {
  SplitGeom g{};
  g.o = o;
  g.v = v;
  g.S = S;
  g.mt = (int)(((long long)v * v + MROWS - 1) / MROWS);
  g.kbv = (v + KB - 1) / KB;
  g.kbo = (o + KB - 1) / KB;
  g.hv = (v + 7) / 8;
  g.ho = (o + 7) / 8;
  const int vp = g.kbv * KB;
  const int ncmax = S >= 4 ? NCMAX_S4 : NCMAX;
  g.nch = (vp + ncmax - 1) / ncmax;
  g.nc = ((vp + g.nch - 1) / g.nch + 15) / 16 * 16;
  g.vc = (v + 3) / 4 * 4;
  // Triplets per block: about 64 W-term items per SM of a 152-SM GPU in each
  // of the block's three W-term launches (fewer, longer launches: less time in
  // launch tails), at most 256, at most a 4 GB W buffer and at most the number
  // of triplets.
  const long long per_trip = (long long)g.mt * g.nch;
  long long nb = (64LL * 152 + per_trip - 1) / per_trip;
  nb = std::min<long long>(nb, (4LL << 30) / ((long long)v * v * g.vc * 4));
  nb = std::max<long long>(1, std::min<long long>(256, nb));
  const long long ntrip = std::max<long long>(1, (long long)o * (o + 1) * (o + 2) / 6 - o);
  g.nb = (int)std::min(nb, ntrip);
  return g;
}

SplitLayout split_layout(int o, int v, int S) {
  SplitLayout L{};
  const SplitGeom g = split_geom(o, v, S);
  L.g = g;
  const size_t a_v = (size_t)o * g.mt * g.hv * S * A_HALF, a_o = (size_t)o * g.mt * g.ho * S * A_HALF;
  const size_t b_v = (size_t)o * o * g.nch * g.hv * S * g.nc * 16, b_o = (size_t)o * o * g.nch * g.ho * S * g.nc * 16;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = (off + bytes + 255) & ~(size_t)255; return r; };
  L.pa = take(a_v);
  L.pa2 = take(a_v);
  L.hc = take(a_o);
  L.hc2 = take(a_o);
  L.tb = take(b_v);
  L.hb = take(b_o);
  L.t1f = take((size_t)o * g.vc * 4);
  L.epsf = take((size_t)2 * (o + v) * 4);
  L.ovovf = take((size_t)2 * o * v * o * g.vc * 4);
  L.y = take((size_t)g.nb * v * v * g.vc * 4);
  L.total = off;
  return L;
}

namespace {
// (half, row) entries of image `kind` per value of its first occupied index.
long long image_per_first(int kind, const SplitGeom &g) {
  const int nh = (kind == 0 || kind == 1 || kind == 4) ? g.hv : g.ho;
  return kind < 4 ? (long long)g.mt * nh * MROWS : (long long)g.o * g.nch * nh * g.nc;
}
constexpr int PREP_BLOCKS = 152 * 16, PREP_THREADS = 256;
}  // namespace

cudaError_t launch_split_prep_common(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st) {
  const SplitGeom &g = L.g;
  unsigned char *b = (unsigned char *)ws;
  f32_rows<<<PREP_BLOCKS, PREP_THREADS, 0, st>>>(in.t1, g.o, g.v, g.vc, (float *)(b + L.t1f));
  f32_hilo<<<PREP_BLOCKS, PREP_THREADS, 0, st>>>(in.eps, g.o + g.v, (float *)(b + L.epsf));
  return cudaGetLastError();
}

cudaError_t launch_split_prep_range(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st, int p0,
                                    int p1) {
  const SplitGeom &g = L.g;
  if (p0 < 0 || p1 > g.o || p0 >= p1) return cudaErrorInvalidValue;
  unsigned char *b = (unsigned char *)ws;
  const size_t off[6] = {L.pa, L.pa2, L.hc, L.hc2, L.tb, L.hb};
  const double *src[6] = {in.ovvv, in.ovvv, in.t2, in.t2, in.t2, in.ovoo};
  for (int kind = 0; kind < 6; ++kind) {
    const long long per = image_per_first(kind, g);
    build_image<<<PREP_BLOCKS, PREP_THREADS, 0, st>>>(kind, src[kind], g, per * p0, per * p1, b + off[kind]);
  }
  ovov_f32<<<PREP_BLOCKS, PREP_THREADS, 0, st>>>(in.ovov, g.o, g.v, g.vc, p0, p1, (float *)(b + L.ovovf));
  return cudaGetLastError();
}

cudaError_t launch_split_prep(const SplitLayout &L, const Inputs &in, void *ws, cudaStream_t st) {
  cudaError_t e = launch_split_prep_common(L, in, ws, st);
  if (e != cudaSuccess) return e;
  return launch_split_prep_range(L, in, ws, st, 0, L.g.o);
}

int split_prep_launches() { return 9; }
int split_prep_range_launches() { return 7; }

WtJob wt_job(const SplitLayout &L, const void *ws, const int4 *trip, int t0, int nt) {
  const unsigned char *b = (const unsigned char *)ws;
  WtJob J{};
  J.g = L.g;
  J.trip = trip;
  J.t0 = t0;
  J.nt = nt;
  J.pa = b + L.pa;
  J.pa2 = b + L.pa2;
  J.hc = b + L.hc;
  J.hc2 = b + L.hc2;
  J.tb = b + L.tb;
  J.hb = b + L.hb;
  J.y = (float *)(b + L.y);
  return J;
}

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (EncodeTiled)p;
  }();
  return fn;
}
}  // namespace

cudaError_t en_job(EnJob *out, const Dims &d, const SplitLayout &L, const void *ws, const Inputs &in, const Work &w,
                   int t0, int nt) {
  const unsigned char *b = (const unsigned char *)ws;
  EnJob &J = *out;
  J = EnJob{};
  J.d = d;
  J.g = L.g;
  J.trip = w.trip;
  J.orb = w.orb;
  J.eps = in.eps;
  J.t1f = (const float *)(b + L.t1f);
  J.epsf = (const float *)(b + L.epsf);
  J.ovovf = (const float *)(b + L.ovovf);
  J.y = (const float *)(b + L.y);
  J.partial = w.partial;
  J.t0 = t0;
  J.nt = nt;
  // W buffer [nt][a][b][vc] as (c < v, b < v, a < v, t): boxes of 16^3,
  // zero-filled where an index reaches v
  const SplitGeom &g = L.g;
  EncodeTiled enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t rowb = (cuuint64_t)g.vc * 4;
  const cuuint64_t dims[4] = {(cuuint64_t)g.v, (cuuint64_t)g.v, (cuuint64_t)g.v, (cuuint64_t)nt};
  const cuuint64_t strides[3] = {rowb, rowb * g.v, rowb * g.v * g.v};
  const cuuint32_t box[4] = {NT, NT, NT, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&J.ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)J.y, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // FP32 (p u|q w) in both orders, [h][x0][x1][x2][vc] as (x3 < v, x2 < o,
  // x1 < v, x0 < o, h): 16 x 16 tiles over (x1, x3)
  const cuuint64_t gdims[5] = {(cuuint64_t)g.v, (cuuint64_t)g.o, (cuuint64_t)g.v, (cuuint64_t)g.o, 2};
  const cuuint64_t gstr[4] = {rowb, rowb * g.o, rowb * g.o * g.v, rowb * g.o * g.v * g.o};
  const cuuint32_t gbox[5] = {NT, 1, NT, 1, 1};
  const cuuint32_t gestr[5] = {1, 1, 1, 1, 1};
  r = enc(&J.gmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, (void *)J.ovovf, gdims, gstr, gbox, gestr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // FP32 t1 [o][vc] as (a < v, i < o): rows of 16
  const cuuint64_t tdims[2] = {(cuuint64_t)g.v, (cuuint64_t)g.o};
  const cuuint64_t tstr[1] = {rowb};
  const cuuint32_t tbox[2] = {NT, 1};
  const cuuint32_t testr[2] = {1, 1};
  r = enc(&J.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)J.t1f, tdims, tstr, tbox, testr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t split_block_params(WtBatch *wb, EnBatch &eb, int S, int num_sms, void **wargs, void **eargs,
                               cudaKernelNodeParams *wp, cudaKernelNodeParams *ep) {
  int wgrid = 1, egrid = 1;
  size_t wsmem = 0;
  WtKernel wfn = nullptr;
  cudaError_t e = prepare(wb[0], eb, S, num_sms, &wgrid, &egrid, &wsmem, &wfn);
  if (e != cudaSuccess) return e;
  for (int f = 0; f < SPLIT_WT_LAUNCHES; ++f) {
    if (f > 0) wb[f] = wb[0];
    for (int j = 0; j < wb[f].njobs; ++j) wb[f].job[j].gsel = f;
    wt_params(wfn, wb[f], wgrid, wsmem, &wargs[f], &wp[f]);
  }
  eargs[0] = (void *)&eb;
  *ep = cudaKernelNodeParams{};
  ep->func = (void *)tc_energy_kernel;
  ep->gridDim = dim3(egrid);
  ep->blockDim = dim3(EN_THREADS);
  ep->sharedMemBytes = EN_SMEM;
  ep->kernelParams = eargs;
  return cudaSuccess;
}

cudaError_t launch_split_block(WtBatch &wb, EnBatch &eb, int S, int num_sms, cudaStream_t st,
                               cudaEvent_t w0, cudaEvent_t w1) {
  int wgrid = 1, egrid = 1;
  size_t wsmem = 0;
  WtKernel wfn = nullptr;
  cudaError_t e = prepare(wb, eb, S, num_sms, &wgrid, &egrid, &wsmem, &wfn);
  if (e != cudaSuccess) return e;
  if (w0 && (e = cudaEventRecord(w0, st)) != cudaSuccess) return e;
  // Programmatic launches: each kernel of the chain may start its CTAs on SMs
  // that the previous one has left and waits (griddepcontrol.wait) for that
  // kernel's completion only before it touches Y.
  cudaLaunchAttribute attr{};
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.stream = st;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(wgrid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = wsmem;
  // F(i,j,k), F(i,k,j), F(j,k,i) in this order (the batch is copied at each launch)
  for (int f = 0; f < SPLIT_WT_LAUNCHES; ++f) {
    for (int j = 0; j < wb.njobs; ++j) wb.job[j].gsel = f;
    e = cudaLaunchKernelEx(&cfg, wfn, wb);
    if (e != cudaSuccess) return e;
  }
  if (w1 && (e = cudaEventRecord(w1, st)) != cudaSuccess) return e;
  cfg.gridDim = dim3(egrid);
  cfg.blockDim = dim3(EN_THREADS);
  cfg.dynamicSmemBytes = EN_SMEM;
  return cudaLaunchKernelEx(&cfg, tc_energy_kernel, eb);
}

}  // namespace tc
