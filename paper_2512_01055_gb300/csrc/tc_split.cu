// Split-precision path: W (Eqs. 2, 5) from BF16 slices on the tcgen05 tensor
// cores (FP32 accumulation in TMEM), V (Eq. 3) in FP32, D (Fig. 4 sign) and
// its reciprocal in FP64, per-item energy sums in FP64.
//
// Slices.  Every FP64 operand x is written as s BF16 numbers x_0 + ... + x_{s-1}
// with x_0 = bf16(x) and x_p = bf16(x - x_0 - ... - x_{p-1}) (round to
// nearest; the FP64 residual is exact), the splitting used to emulate higher
// precision with BF16 products (Henry, Tang, Heinecke, ARITH 2019; an
// Ozaki-style error-free-ish expansion with per-element exponents).  A product
// is approximated by the slice pairs with p + q < s, grouped by level L = p + q.
//
// GEMM tiles.  Virtual tiles have edge 16.  A "job" is one A tile of 256 rows
// (pairs of two virtual tiles) and one or two B panels of 16 rows:
//   particle:  A = (x a | b f) = ovvv[x][a][b][f],  B = t2[y][z][c][f],  K = v
//   hole:      A = t2[l][z][a][b] (re-laid out with l last),  B = -(x c | y l),  K = o
// For each K step of 16 the MMA warp issues, per 128-row half, one MMA per A
// slice p with the B slices 0 .. s-1-p stacked along N, so each A slice is read
// from shared memory once and lands in its level's TMEM columns.  The drain
// warps add the levels (smallest first) and scatter the 256 x 16 (x panels)
// results into the orbit's W blocks in shared memory with the job's index
// permutation.  After all jobs of an orbit, the same warps evaluate the Eq. 1
// bracket over the orbit's canonical points (as in the FP64 path) and
// accumulate FP64 partials.
//
// Operand images.  The slicer writes every A tile (256 rows x 16 K) and B
// panel (16 rows x 16 K) of every K block directly in the tensor core's
// K-major no-swizzle layout (8-row x 16-byte core matrices, the two K halves
// 128 bytes apart, 8-row groups 256 bytes apart), tile-major with the S slices
// of a block contiguous.  One pipeline stage is then one contiguous bulk copy
// (cp.async.bulk) for A and one per B slice, instead of hundreds of 32-byte
// tensor-map rows per stage.
//
// Warp roles (320 threads): warp 0 issues the bulk copies, warp 1 owns TMEM
// and lane 0 issues MMAs, warps 2-9 (two warpgroups, one per 128-row half of
// each job) drain TMEM and run the energy epilogue.
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// lets every role leave its loop, waits (bounded) for its own copies and MMAs
// and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int NT = 16;                    // virtual tile edge
constexpr int KC = 16;                    // K per pipeline stage (32-byte rows, 32B swizzle)
constexpr int A_SLICE_BYTES = 256 * KC * 2;
constexpr int B_PANEL_BYTES = NT * KC * 2;
constexpr int MAXS = 4;
constexpr int MAX_STAGES = 8;
// Copy issue: one warp completes about one pipeline stage per ~0.36 us however
// many stages it has in flight, while several issuing warps overlap.  NPROD
// producer warps (warp 0 and warps 10, 11, ...) therefore fill the stages
// round-robin.
// MMA issue: one issuing thread spends ~210 ns on the six MMAs of a K block
// (N = 96, 64, 32 per half); two issuing warps, one per 128-row half of the A
// tile, bring it to ~150 ns.  Warp 1 issues half 0 and warp 12 half 1.
constexpr int NPROD = 3;
constexpr int MMA_WARP1 = 10 + (NPROD - 1);
constexpr int THREADS = 32 * (MMA_WARP1 + 1);
constexpr int EPI_THREADS = 256;
constexpr int EPI_WARPS = EPI_THREADS / 32;
constexpr int WX = 273, WY = 17;          // W block index = x*WX + y*WY + z (bank-friendly)
constexpr int WBLK = 4368;                // floats per W block (>= 15*WX + 15*WY + 16)
constexpr int W_BYTES = 6 * WBLK * 4;
constexpr int MAX_JOBS = 72;
constexpr long long WAIT_LIMIT = 1LL << 26;
// Longest run of K blocks accumulated in one tensor-core accumulator.  The FP32
// accumulation along K rounds systematically, so longer products are split into
// chains of at most KCHAIN blocks (256 K values), each drained and added into W.
constexpr int KCHAIN = 16;

constexpr int ERR_TIMEOUT_FULL = 11, ERR_TIMEOUT_EMPTY = 12, ERR_TIMEOUT_ACCFULL = 13,
              ERR_TIMEOUT_ACCEMPTY = 14, ERR_TIMEOUT_TEARDOWN = 15;

// One GEMM job of an (occupied pattern, tile pattern) template.  Every field
// is a position (0, 1, 2) into the triplet's occupied indices occ[] or the
// orbit's tile indices tl[], so one template serves every triplet and orbit
// with the same equality pattern (i > j > k, i = j > k, i > j = k) x
// (P > Q > R, P = Q > R, P > Q = R, P = Q = R).
struct TJob {
  uint8_t kind;              // 0 particle, 1 hole
  uint8_t np;                // panels (1 or 2)
  uint8_t apos;              // A tile occupied index: occ[apos]
  uint8_t tapos, tbpos;      // A rows (a, b): a in tile tl[tapos], b in tile tl[tbpos]
  uint8_t pad;
  uint8_t ptpos[2];          // panel tile tl[ptpos]
  uint8_t p0pos[2];          // particle: y of t2[y][z]; hole: x of (x c|y l)
  uint8_t p1pos[2];          // particle: z;              hole: y
  uint8_t blk[2];            // W block (distinct permutation index of the orbit)
  uint8_t hi[2], lo[2], col[2];   // W positions receiving row/16, row%16 and the panel column
};
constexpr int N_PATTERNS = 12;
__constant__ TJob c_tjobs[N_PATTERNS][MAX_JOBS];
__constant__ int c_ntjobs[N_PATTERNS];

__host__ __device__ __forceinline__ int pattern_id(const int occ[3], const int tl[3]) {
  const int op = (occ[0] == occ[1]) ? 1 : ((occ[1] == occ[2]) ? 2 : 0);
  const int tp = (tl[0] == tl[1] && tl[1] == tl[2]) ? 3 : ((tl[0] == tl[1]) ? 1 : ((tl[1] == tl[2]) ? 2 : 0));
  return op * 4 + tp;
}


__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}

// Bounded wait; gives up early when another role has aborted.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *err, int code) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 255) == 255) {
      if (*abort_flag) return false;
      __nanosleep(128);
    }
  }
  *abort_flag = 1;
  atomicCAS(err, 0, code);
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle; core matrices of 8 rows
// x 16 bytes, the next core matrix along K 128 bytes on, the next 8-row group
// 256 bytes on.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;                 // leading byte offset (K direction)
  d |= (uint64_t)(256 >> 4) << 32;                 // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                          // descriptor version
  return d;                                        // swizzle field 0
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dcol, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               :: "r"(dcol), "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" :: "n"(EPI_THREADS) : "memory"); }
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

// The GEMM jobs of one (triplet, orbit) pattern: for every distinct block s and
// every permutation u of Eq. 5, one particle and one hole product; products
// that share an A tile are paired into one job (at most two panels).  Built on
// the host from representative index values; positions are stored.
int host_build_template(const int occ[3], const int tl[3], TJob *jobs) {
  auto opos = [&](int val) { return val == occ[0] ? 0 : (val == occ[1] ? 1 : 2); };
  auto tpos = [&](int val) { return val == tl[0] ? 0 : (val == tl[1] ? 1 : 2); };
  int blk[6];
  orbit_blocks(tl, blk);
  int n = 0;
  for (int kind = 0; kind < 2; ++kind) {
    const int first = n;
    for (int s = 0; s < 6; ++s) {
      if (blk[s] != s) continue;
      int T[3];
      for (int p = 0; p < 3; ++p) T[p] = tl[perm3(s, p)];
      for (int u = 0; u < 6; ++u) {
        const int u0 = perm3(u, 0), u1 = perm3(u, 1), u2 = perm3(u, 2);
        int aocc, ta, tb, ptile, po0, po1, hi, lo, col;
        if (kind == 0) {   // sum_f (x p | q f) t2[z][y][r][f]: rows (u0, u1), column u2
          aocc = occ[u0]; ta = T[u0]; tb = T[u1];
          ptile = T[u2]; po0 = occ[u2]; po1 = occ[u1];
          hi = u0; lo = u1; col = u2;
        } else {           // -sum_l (x p | y l) t2[l][z][q][r]: rows (u1, u2), column u0
          aocc = occ[u2]; ta = T[u1]; tb = T[u2];
          ptile = T[u0]; po0 = occ[u0]; po1 = occ[u1];
          hi = u1; lo = u2; col = u0;
        }
        int j = -1;
        for (int q = first; q < n; ++q)
          if (jobs[q].np == 1 && occ[jobs[q].apos] == aocc && tl[jobs[q].tapos] == ta && tl[jobs[q].tbpos] == tb) {
            j = q;
            break;
          }
        int slot = 1;
        if (j < 0) {
          j = n++;
          jobs[j] = TJob{};
          jobs[j].kind = (uint8_t)kind;
          jobs[j].apos = (uint8_t)opos(aocc);
          jobs[j].tapos = (uint8_t)tpos(ta);
          jobs[j].tbpos = (uint8_t)tpos(tb);
          slot = 0;
        }
        jobs[j].np = (uint8_t)(slot + 1);
        jobs[j].ptpos[slot] = (uint8_t)tpos(ptile);
        jobs[j].p0pos[slot] = (uint8_t)opos(po0);
        jobs[j].p1pos[slot] = (uint8_t)opos(po1);
        jobs[j].blk[slot] = (uint8_t)s;
        jobs[j].hi[slot] = (uint8_t)hi; jobs[j].lo[slot] = (uint8_t)lo; jobs[j].col[slot] = (uint8_t)col;
      }
    }
  }
  return n;
}

template <int S>
__global__ void __launch_bounds__(THREADS, 1)
tc_split_kernel(const __grid_constant__ SplitBatch B) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int STAGE_BYTES = S * (A_SLICE_BYTES + 2 * B_PANEL_BYTES);
  float *Wsm = (float *)(sm + B.stages * STAGE_BYTES);

  __shared__ __align__(8) uint64_t full_bar[MAX_STAGES], empty_bar[MAX_STAGES];
  __shared__ __align__(8) uint64_t accfull_bar[2], accempty_bar[2], teardown_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int abort_flag;
  __shared__ int epi_ok;
  __shared__ double red[EPI_WARPS];
  __shared__ long long last_seq[NPROD][MAX_STAGES];   // per producer: its latest copy into each stage

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid < NPROD * MAX_STAGES) last_seq[tid / MAX_STAGES][tid % MAX_STAGES] = -1;
  if (tid == 0) {
    // a stage is free, and an accumulator buffer full, once both MMA warps committed
    for (int s = 0; s < B.stages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 2); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accfull_bar[b], 2); mbar_init(&accempty_bar[b], 1); }
    mbar_init(&teardown_bar[0], 1);
    mbar_init(&teardown_bar[1], 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base_sh)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (warp >= 2 && warp < 10) {
    for (int e = tid - 64; e < 6 * WBLK; e += EPI_THREADS) Wsm[e] = 0.f;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base_sh;
  constexpr int BUFCOLS = 2 * S * 32;

  if (warp == 0 || (warp >= 10 && warp < MMA_WARP1)) {
    // ------------------------------------------------------------ bulk-copy producers (whole warps)
    // Every producer walks the same sequence of K blocks; producer pw fills the
    // blocks whose sequence number is pw modulo NPROD.
    const int pw = warp == 0 ? 0 : warp - 9;
    int stage = 0;
    uint32_t phase = 0;
    long long seq = 0;
    int rr = 0;                               // seq modulo NPROD
    bool ok = true;
    int jc = 0;
    for (long long gitem = blockIdx.x; ok && gitem < B.total_items; gitem += gridDim.x) {
      while (jc + 1 < B.njobs && gitem >= B.job[jc + 1].item0) ++jc;   // items ascend: the cursor only moves on
      const SplitJob &P = B.job[jc];
      const Dims &d = P.d;
      const int o = d.o, v = d.v;
      const long long item = gitem - P.item0 + P.item_base;
      (void)v;
      int t, chunk;
      item_slot(d, item, t, chunk);
      const int4 tr = P.w.trip[t];
      const int occ[3] = {tr.x, tr.y, tr.z};
      const int ob1 = min(d.n_orb, (chunk + 1) * d.orb_per_item);
      for (int ob = chunk * d.orb_per_item; ok && ob < ob1; ++ob) {
        const int4 og = P.w.orb[ob];
        const int tl[3] = {og.x, og.y, og.z};
        const int pid = pattern_id(occ, tl);
        const int nj = c_ntjobs[pid];
        for (int jb = 0; ok && jb < nj; ++jb) {
          const TJob J = c_tjobs[pid][jb];
          const int np = J.np;
          const int nk = J.kind == 0 ? P.kch_p : P.kch_h;
          const uint32_t bytes = (uint32_t)S * (A_SLICE_BYTES + np * B_PANEL_BYTES);
          const int aocc = occ[J.apos], ta = tl[J.tapos], tb = tl[J.tbpos];
          const int T = P.T;
          // A image of K block kc: ((aocc*T + ta)*T + tb)*nk + kc, S slices of 8 KB each
          const unsigned char *srcA = (J.kind == 0 ? P.imgA_p : P.imgA_h) +
                                      ((size_t)((aocc * T + ta) * T + tb) * nk) * S * A_SLICE_BYTES;
          // lane 1 + (q * 2 + pn) copies B slice q of panel pn
          const int bl = lane - 1, bq = bl / 2, bpn = bl % 2;
          const bool bload = lane >= 1 && bq < S && bpn < np;
          const unsigned char *srcB = nullptr;
          if (bload) {
            const int bt = tl[J.ptpos[bpn]], b0 = occ[J.p0pos[bpn]], b1 = occ[J.p1pos[bpn]];
            srcB = (J.kind == 0 ? P.imgB_p : P.imgB_h) + ((size_t)((b0 * o + b1) * T + bt) * nk * S + bq) * B_PANEL_BYTES;
          }
          for (int kc = 0; kc < nk; ++kc, ++seq) {
            const bool mine = rr == pw;
            if (++rr == NPROD) rr = 0;
            if (mine) {
              int got = 1;
              if (lane == 0) {
                got = mbar_wait(&empty_bar[stage], phase ^ 1u, &abort_flag, B.err, ERR_TIMEOUT_EMPTY) ? 1 : 0;
                if (got) {
                  last_seq[pw][stage] = seq;
                  mbar_expect_tx(&full_bar[stage], bytes);
                }
              }
              got = __shfl_sync(0xffffffffu, got, 0);
              if (!got) { ok = false; break; }
              unsigned char *sA = sm + stage * STAGE_BYTES;
              unsigned char *sB = sA + S * A_SLICE_BYTES;
              if (lane == 0) {
                bulk_load(sA, srcA + (size_t)kc * S * A_SLICE_BYTES, S * A_SLICE_BYTES, &full_bar[stage]);
              } else if (bload) {
                bulk_load(sB + (bq * np + bpn) * B_PANEL_BYTES, srcB + (size_t)kc * S * B_PANEL_BYTES, B_PANEL_BYTES,
                          &full_bar[stage]);
              }
              __syncwarp();
            }
            if (++stage == B.stages) { stage = 0; phase ^= 1u; }
          }
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
  } else if (warp == 1 || warp == MMA_WARP1) {
    // ------------------------------------------------------------ MMA issuers, one per 128-row half
    const int mh = warp == 1 ? 0 : 1;
    if (lane == 0) {
      int stage = 0, abuf = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      int jc = 0;
    for (long long gitem = blockIdx.x; ok && gitem < B.total_items; gitem += gridDim.x) {
      while (jc + 1 < B.njobs && gitem >= B.job[jc + 1].item0) ++jc;   // items ascend: the cursor only moves on
      const SplitJob &P = B.job[jc];
      const Dims &d = P.d;
      const int o = d.o, v = d.v;
      const long long item = gitem - P.item0 + P.item_base;
      (void)v;
        int t, chunk;
        item_slot(d, item, t, chunk);
        const int4 tr = P.w.trip[t];
        const int occ[3] = {tr.x, tr.y, tr.z};
        const int ob1 = min(d.n_orb, (chunk + 1) * d.orb_per_item);
        for (int ob = chunk * d.orb_per_item; ok && ob < ob1; ++ob) {
          const int4 og = P.w.orb[ob];
          const int tl[3] = {og.x, og.y, og.z};
          const int pid = pattern_id(occ, tl);
          const int nj = c_ntjobs[pid];
          for (int jb = 0; ok && jb < nj; ++jb) {
            const int np = c_tjobs[pid][jb].np;
            const int nk = c_tjobs[pid][jb].kind == 0 ? P.kch_p : P.kch_h;
            const int nchain = (nk + KCHAIN - 1) / KCHAIN;
            for (int ch = 0; ok && ch < nchain; ++ch) {
            const int kc0 = ch * nk / nchain, kc1 = (ch + 1) * nk / nchain;
            if (!mbar_wait(&accempty_bar[abuf], aphase ^ 1u, &abort_flag, B.err, ERR_TIMEOUT_ACCEMPTY)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t dbase = tbase + (uint32_t)(abuf * BUFCOLS);
            for (int kc = kc0; kc < kc1; ++kc) {
              if (!mbar_wait(&full_bar[stage], phase, &abort_flag, B.err, ERR_TIMEOUT_FULL)) { ok = false; break; }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              const uint32_t sA = smem_u32(sm + stage * STAGE_BYTES);
              const uint64_t bd = sdesc(sA + S * A_SLICE_BYTES);
#pragma unroll
              for (int a = 0; a < S; ++a) {
                const uint64_t ad = sdesc(sA + a * A_SLICE_BYTES + mh * (A_SLICE_BYTES / 2));
                const uint32_t dcol = dbase + (uint32_t)(mh * S * 32 + a * np * NT);
                mma_bf16(dcol, ad, bd, idesc(128, (S - a) * np * NT), (kc > kc0 || a > 0) ? 1u : 0u);
              }
              mma_commit(&empty_bar[stage]);
              if (++stage == B.stages) { stage = 0; phase ^= 1u; }
            }
            if (!ok) break;
            mma_commit(&accfull_bar[abuf]);
            if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
            }
          }
        }
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(&teardown_bar[mh]);
      const uint32_t a = smem_u32(&teardown_bar[mh]);
      for (long long it = 0; it < WAIT_LIMIT && !mbar_try(a, 0); ++it) {
        if ((it & 255) == 255) __nanosleep(128);
        if (it == WAIT_LIMIT - 1) atomicCAS(B.err, 0, ERR_TIMEOUT_TEARDOWN);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ drain + energy epilogue
    const int et = tid - 64;                  // 0 .. 255
    const int quarter = warp & 3;             // TMEM lane quarter this warp may access
    const int lrow = 32 * quarter + lane;     // row within a 128-row half
    const int h = et >> 7;                    // warpgroup -> 128-row half of every job
    int abuf = 0;
    uint32_t aphase = 0;
    bool ok = true;
    int jc = 0;
    for (long long gitem = blockIdx.x; ok && gitem < B.total_items; gitem += gridDim.x) {
      while (jc + 1 < B.njobs && gitem >= B.job[jc + 1].item0) ++jc;   // items ascend: the cursor only moves on
      const SplitJob &P = B.job[jc];
      const Dims &d = P.d;
      const int o = d.o, v = d.v;
      const long long item = gitem - P.item0 + P.item_base;
      (void)v;
      int t, chunk;
      const long long islot = item_slot(d, item, t, chunk);
      const int4 tr = P.w.trip[t];
      const int occ[3] = {tr.x, tr.y, tr.z};
      const double eijk = __ldg(P.eps + occ[0]) + __ldg(P.eps + occ[1]) + __ldg(P.eps + occ[2]);
      double acc = 0.0;
      const int ob1 = min(d.n_orb, (chunk + 1) * d.orb_per_item);
      for (int ob = chunk * d.orb_per_item; ok && ob < ob1; ++ob) {
        const int4 og = P.w.orb[ob];
        const int tl[3] = {og.x, og.y, og.z};
        const int pid = pattern_id(occ, tl);
        const int nj = c_ntjobs[pid];
        for (int jb = 0; jb < nj; ++jb) {
          const TJob J = c_tjobs[pid][jb];
          const int nchain = ((J.kind == 0 ? P.kch_p : P.kch_h) + KCHAIN - 1) / KCHAIN;
          for (int ch = 0; ch < nchain; ++ch) {
          if (et == 0)
            epi_ok = mbar_wait(&accfull_bar[abuf], aphase, &abort_flag, B.err, ERR_TIMEOUT_ACCFULL) ? 1 : 0;
          epi_bar();
          if (!epi_ok) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t dbase = tbase + (uint32_t)(abuf * BUFCOLS) + ((uint32_t)(32 * quarter) << 16);
          const int np = J.np;
          // The two panels of a job may update the same W elements (coincident tiles put
          // both products in one block with different orientations), so panel 1 starts
          // only after every thread has finished panel 0.
#pragma unroll
          for (int pn = 0; pn < 2; ++pn) {
            if (pn >= np) break;
            if (pn == 1) epi_bar();
            {
              const int row = h * 128 + lrow;
              const int rhi = row >> 4, rlo = row & 15;
              float lv[S][16];
#pragma unroll
              for (int L = 0; L < S; ++L) tmem_ld16(dbase + (uint32_t)(h * S * 32 + L * np * NT + pn * NT), lv[L]);
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
              int lc[3];
              lc[J.hi[pn]] = rhi;
              lc[J.lo[pn]] = rlo;
              lc[J.col[pn]] = 0;
              const int cstride = (J.col[pn] == 0) ? WX : (J.col[pn] == 1 ? WY : 1);
              float *base = Wsm + J.blk[pn] * WBLK + lc[0] * WX + lc[1] * WY + lc[2];
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                float sum = lv[S - 1][j];             // smallest level first
#pragma unroll
                for (int L = S - 2; L >= 0; --L) sum += lv[L][j];
                base[j * cstride] += sum;
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          epi_bar();                             // all loads and W updates of this job are done
          if (et == 0) mbar_arrive(&accempty_bar[abuf]);
          if (++abuf == 2) { abuf = 0; aphase ^= 1u; }
          }
          if (!ok) break;
        }
        if (!ok) break;

        // energy over the canonical points a >= b >= c of the orbit
        int blk[6];
        orbit_blocks(tl, blk);
        for (int pr = et; pr < NT * NT; pr += EPI_THREADS) {
          const int la = pr >> 4, lb = pr & 15;
          const int ga = tl[0] * NT + la, gb = tl[1] * NT + lb;
          if (ga >= v || gb >= v || ga < gb) continue;
          const double dab = eijk - (__ldg(P.eps + o + ga) + __ldg(P.eps + o + gb));
          for (int lcc = 0; lcc < NT; ++lcc) {
            const int gc = tl[2] * NT + lcc;
            if (gc >= v || gb < gc) continue;
            const int l3[3] = {la, lb, lcc};
            const int g[3] = {ga, gb, gc};
            float ws[6], vs[6];
#pragma unroll
            for (int s = 0; s < 6; ++s) {
              const int p0 = perm3(s, 0), p1 = perm3(s, 1), p2 = perm3(s, 2);
              ws[s] = Wsm[blk[s] * WBLK + l3[p0] * WX + l3[p1] * WY + l3[p2]];
              const int x = g[p0], y = g[p1], z = g[p2];
              const float *ov = P.ovovf;
              vs[s] = __ldg(P.t1f + occ[0] * v + x) * __ldg(ov + ((occ[1] * v + y) * o + occ[2]) * v + z)
                    + __ldg(P.t1f + occ[1] * v + y) * __ldg(ov + ((occ[0] * v + x) * o + occ[2]) * v + z)
                    + __ldg(P.t1f + occ[2] * v + z) * __ldg(ov + ((occ[0] * v + x) * o + occ[1]) * v + y);
            }
            const float se = ws[0] + ws[3] + ws[4];
            const float so = ws[1] + ws[2] + ws[5];
            float sum = 0.f;
#pragma unroll
            for (int s = 0; s < 6; ++s) {
              const float br = 3.f * ws[s] + (perm3_even(s) ? se - 2.f * so : so - 2.f * se);
              sum = fmaf(ws[s] + vs[s], br, sum);
            }
            // FP64 denominator: D = e_i + e_j + e_k - e_a - e_b - e_c and 1/D by one
            // Newton-Raphson step from the hardware reciprocal estimate.
            const double D = dab - __ldg(P.eps + o + gc);
            double r;
            asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(D));
            r = fma(r, fma(-D, r, 1.0), r);
            const double mult = (ga == gc) ? (1.0 / 6.0) : ((ga == gb || gb == gc) ? 0.5 : 1.0);
            acc = fma((double)sum * mult, r, acc);
          }
        }
        epi_bar();
        for (int e = et; e < 6 * WBLK; e += EPI_THREADS) Wsm[e] = 0.f;
        epi_bar();
      }
      if (!ok) break;
      // the item's partial: fixed-order reduction over the 128 epilogue threads
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) red[warp - 2] = acc;
      epi_bar();
      if (et == 0) {
        double tot = 0.0;
#pragma unroll
        for (int wq = 0; wq < EPI_WARPS; ++wq) tot += red[wq];
        P.w.partial[islot] = tot;
      }
      epi_bar();
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512));
  }
}

// ---------------------------------------------------------------- operand images

// One thread per (image, row, K half): reads 8 consecutive K values of one
// operand row, splits them into S BF16 slices and writes 16 bytes per slice at
// the row's place in the no-swizzle K-major image.  Rows or K values outside
// the tensor are zero.
//   mode 0: A particle  image (x, ta, tb, kb), row (a, b), K = f:  (x a | b f)
//   mode 1: A hole      image (z, ta, tb, kb), row (a, b), K = l:  t2[l][z][a][b]
//   mode 2: B particle  image (y, z, tc, kb),  row c,      K = f:  t2[y][z][c][f]
//   mode 3: B hole      image (x, y, tc, kb),  row c,      K = l:  -(x c | y l)
__global__ void build_images(int mode, const double *__restrict__ src, int o, int v, int T, int nkb, int S,
                             unsigned char *__restrict__ out) {
  const int rows = (mode < 2) ? 256 : 16;
  const int img_bytes = rows * KC * 2;
  const long long nimg = (long long)((mode == 0 || mode == 1) ? o * T * T : o * o * T) * nkb;
  const long long total = nimg * rows * 2;
  const long long vv = (long long)v * v;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int kh = (int)(e & 1);
    const int r = (int)((e >> 1) % rows);
    const long long img = (e >> 1) / rows;
    const int kb = (int)(img % nkb);
    const long long rest = img / nkb;                      // (.., .., tile) or (.., tile, tile)
    double x[8];
    int k0 = kb * KC + kh * 8;
    if (mode < 2) {
      const int tb = (int)(rest % T), ta = (int)((rest / T) % T), xo = (int)(rest / ((long long)T * T));
      const int a = ta * NT + r / NT, b = tb * NT + r % NT;
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        double val = 0.0;
        if (mode == 0) { if (a < v && b < v && k < v) val = src[((long long)xo * v + a) * vv + (long long)b * v + k]; }
        else           { if (a < v && b < v && k < o) val = src[((long long)k * o + xo) * vv + (long long)a * v + b]; }
        x[q] = val;
      }
    } else {
      const int tc = (int)(rest % T);
      const long long pair = rest / T;                     // y*o + z  or  x*o + y
      const int p0 = (int)(pair / o), p1 = (int)(pair % o);
      const int c = tc * NT + r;
      for (int q = 0; q < 8; ++q) {
        const int k = k0 + q;
        double val = 0.0;
        if (mode == 2) { if (c < v && k < v) val = src[(((long long)p0 * o + p1) * v + c) * v + k]; }
        else           { if (c < v && k < o) val = -src[(((long long)p0 * v + c) * o + p1) * o + k]; }
        x[q] = val;
      }
    }
    // position of (row r, K half kh) in the image: core matrix (r/8, kh), row r%8
    const int off = ((r >> 3) * 2 + kh) * 128 + (r & 7) * 16;
    unsigned char *base = out + (size_t)img * S * img_bytes + off;
    for (int p = 0; p < S; ++p) {
      __align__(16) __nv_bfloat16 b16[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        b16[q] = __double2bfloat16(x[q]);
        x[q] -= (double)__bfloat162float(b16[q]);        // exact FP64 residual
      }
      *(uint4 *)(base + (size_t)p * img_bytes) = *(const uint4 *)b16;
    }
  }
}

__global__ void to_f32(const double *__restrict__ in, long long n, float *__restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

int stages_for(int S) {
  const int stage_bytes = S * (A_SLICE_BYTES + 2 * B_PANEL_BYTES);
  const int budget = 227 * 1024 - W_BYTES - 1024 - 256;
  int st = budget / stage_bytes;
  if (st > MAX_STAGES) st = MAX_STAGES;
  // The producers' parity waits on the empty barriers stay unambiguous only
  // while a producer can be at most one ring cycle ahead of the stage's last
  // use, which the in-order MMA consumer guarantees when stages >= NPROD.
  static_assert((227 * 1024 - W_BYTES - 1024 - 256) / (MAXS * (A_SLICE_BYTES + 2 * B_PANEL_BYTES)) >= NPROD,
                "fewer pipeline stages than producer warps");
  return st;
}

size_t smem_for(int S) {
  return (size_t)stages_for(S) * S * (A_SLICE_BYTES + 2 * B_PANEL_BYTES) + W_BYTES + 1024;
}

template <int S>
cudaError_t launch_kernel(long long grid, size_t smem, cudaStream_t st, const SplitBatch &b) {
  cudaError_t e = cudaFuncSetAttribute(tc_split_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_split_kernel<S><<<(int)grid, THREADS, smem, st>>>(b);
  return cudaGetLastError();
}

// The 12 job templates, built on the host once and copied to constant memory
// once per device.
cudaError_t upload_templates(cudaStream_t st) {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  static TJob h[N_PATTERNS][MAX_JOBS];
  static int hn[N_PATTERNS];
  const int occ_rep[3][3] = {{2, 1, 0}, {1, 1, 0}, {1, 0, 0}};
  const int tl_rep[4][3] = {{2, 1, 0}, {1, 1, 0}, {1, 0, 0}, {0, 0, 0}};
  for (int op = 0; op < 3; ++op)
    for (int tp = 0; tp < 4; ++tp) {
      const int pid = pattern_id(occ_rep[op], tl_rep[tp]);
      hn[pid] = host_build_template(occ_rep[op], tl_rep[tp], h[pid]);
    }
  e = cudaMemcpyToSymbolAsync(c_tjobs, h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_ntjobs, hn, sizeof(hn), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

}  // namespace

int split_tile() { return NT; }

SplitLayout split_layout(int o, int v, int S) {
  SplitLayout L{};
  const long long T = (v + NT - 1) / NT, nkb = (v + KC - 1) / KC, nko = (o + KC - 1) / KC;
  L.vpad = (int)(T * NT);
  L.opad = (int)(nko * KC);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off = (off + bytes + 255) & ~(size_t)255; return r; };
  L.ovvv = take((size_t)o * T * T * nkb * S * A_SLICE_BYTES);     // A particle images
  L.t2h = take((size_t)o * T * T * nko * S * A_SLICE_BYTES);      // A hole images
  L.t2 = take((size_t)o * o * T * nkb * S * B_PANEL_BYTES);       // B particle images
  L.ovoo = take((size_t)o * o * T * nko * S * B_PANEL_BYTES);     // B hole images
  L.t1f = take((size_t)o * v * 4);
  L.ovovf = take((size_t)o * v * o * v * 4);
  L.total = off;
  return L;
}

cudaError_t launch_split_prep(const Dims &d, int S, const Inputs &in, void *ws, const SplitLayout &L, cudaStream_t st) {
  const int o = d.o, v = d.v;
  const int T = (v + NT - 1) / NT, nkb = (v + KC - 1) / KC, nko = (o + KC - 1) / KC;
  unsigned char *b = (unsigned char *)ws;
  const int blocks = 152 * 16, thr = 256;
  build_images<<<blocks, thr, 0, st>>>(0, in.ovvv, o, v, T, nkb, S, b + L.ovvv);
  build_images<<<blocks, thr, 0, st>>>(1, in.t2, o, v, T, nko, S, b + L.t2h);
  build_images<<<blocks, thr, 0, st>>>(2, in.t2, o, v, T, nkb, S, b + L.t2);
  build_images<<<blocks, thr, 0, st>>>(3, in.ovoo, o, v, T, nko, S, b + L.ovoo);
  to_f32<<<blocks, thr, 0, st>>>(in.t1, (long long)o * v, (float *)(b + L.t1f));
  to_f32<<<blocks, thr, 0, st>>>(in.ovov, (long long)o * v * o * v, (float *)(b + L.ovovf));
  return cudaGetLastError();
}

SplitJob split_job(const Dims &d, const Inputs &in, const void *ws, const SplitLayout &L, const Work &w) {
  const int o = d.o, v = d.v;
  const unsigned char *b = (const unsigned char *)ws;
  SplitJob P{};
  P.d = d;
  P.kch_p = (v + KC - 1) / KC;
  P.kch_h = (o + KC - 1) / KC;
  P.T = (v + NT - 1) / NT;
  P.imgA_p = b + L.ovvv;
  P.imgA_h = b + L.t2h;
  P.imgB_p = b + L.t2;
  P.imgB_h = b + L.ovoo;
  P.t1f = (const float *)(b + L.t1f);
  P.ovovf = (const float *)(b + L.ovovf);
  P.eps = in.eps;
  P.w = w;
  return P;
}

// Launch one persistent kernel over the batch's items (item0 and total_items
// are filled in here from the jobs' item counts).
template <int S>
void node_params(const SplitBatch &b, int grid, void **args, cudaKernelNodeParams *p) {
  args[0] = (void *)&b;
  *p = cudaKernelNodeParams{};
  p->func = (void *)tc_split_kernel<S>;
  p->gridDim = dim3(grid);
  p->blockDim = dim3(THREADS);
  p->sharedMemBytes = (unsigned)smem_for(S);
  p->kernelParams = args;
}

cudaError_t split_node_params(SplitBatch &b, int S, int grid, void **args, cudaKernelNodeParams *p, cudaStream_t st) {
  if (S < 2 || S > MAXS || b.njobs < 1 || b.njobs > MAX_BATCH) return cudaErrorInvalidValue;
  long long total = 0;
  for (int j = 0; j < b.njobs; ++j) {
    b.job[j].item0 = total;
    total += b.job[j].n_run > 0 ? b.job[j].n_run : b.job[j].d.n_items;
  }
  b.total_items = total;
  b.stages = stages_for(S);
  cudaError_t e = upload_templates(st);
  if (e != cudaSuccess) return e;
  const size_t smem = smem_for(S);
  switch (S) {
    case 2: e = cudaFuncSetAttribute(tc_split_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            node_params<2>(b, grid, args, p); break;
    case 3: e = cudaFuncSetAttribute(tc_split_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            node_params<3>(b, grid, args, p); break;
    default: e = cudaFuncSetAttribute(tc_split_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
             node_params<4>(b, grid, args, p); break;
  }
  return e;
}

cudaError_t launch_split(SplitBatch &b, int S, int num_sms, cudaStream_t st) {
  if (S < 2 || S > MAXS || b.njobs < 1 || b.njobs > MAX_BATCH) return cudaErrorInvalidValue;
  long long total = 0;
  for (int j = 0; j < b.njobs; ++j) {
    b.job[j].item0 = total;
    total += b.job[j].n_run > 0 ? b.job[j].n_run : b.job[j].d.n_items;
  }
  b.total_items = total;
  b.stages = stages_for(S);
  const size_t smem = smem_for(S);
  cudaError_t e = upload_templates(st);
  if (e != cudaSuccess) return e;
  long long grid = num_sms;
  if (grid > total) grid = total;
  if (grid < 1) return cudaSuccess;
  switch (S) {
    case 2: e = launch_kernel<2>(grid, smem, st, b); break;
    case 3: e = launch_kernel<3>(grid, smem, st, b); break;
    default: e = launch_kernel<4>(grid, smem, st, b); break;
  }
  return e;
}

}  // namespace tc
