// tc_energy_dev_noalloc: the FP64 (T) energy for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// runtime which owns every device allocation (a pre-sized memory pool, an
// embedded solver, a plugin that must not disturb its host's allocator), or
// code running where a new allocation could fail or fragment memory at a bad
// moment.  This entry point runs the same FP64 kernels as tc_energy_dev but
// keeps all of its scratch (work tables, per-item partial sums, per-triplet
// sums, the work counter) in one file-scope __device__ array of fixed size,
// so it needs no context and performs no device allocation of its own.
//
// The array is part of the library's device image: every GPU that loads the
// library holds TC_NOALLOC_SCRATCH_BYTES of it until the process exits.
// Every call shares it and it keeps the last call's contents; the work
// counter is cleared on every call, and the partial sums are overwritten
// before they are read.  Two calls whose GPU work overlaps (different streams,
// or different host threads) race on the array; callers must serialise them.
//
// In host code the array's name denotes a host-side stand-in, not a device
// address, so host code never passes it to a kernel: the first call on each
// device (with that device current) looks up the device address with
// cudaGetSymbolAddress and caches it.  That first call also sets the fused
// kernel's shared-memory attribute, so it should come before any stream
// capture.  The cached address belongs to the device's primary context: it
// is valid while that context lives, i.e. as long as nobody resets the device
// (cudaDeviceReset) and the caller runs in the runtime's primary context.
#include <cstdio>
#include <mutex>

#include "../../include/tc.h"
#include "tc_internal.cuh"

namespace {

constexpr size_t kScratchBytes = TC_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceSetup {
  bool ready = false;
  unsigned char *scratch = nullptr;   // device address of g_noalloc_scratch on this device
  int num_sms = 0;
  int blocks_per_sm = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Carve {
  size_t trip, orb, partial, e_trip, out, counter, total;
};

Carve carve(const tc::Dims &d) {
  Carve c{};
  size_t off = 0;
  c.trip = off;    off = al256(off + sizeof(int4) * (size_t)(d.n_trip > 0 ? d.n_trip : 1));
  c.orb = off;     off = al256(off + sizeof(int4) * (size_t)d.n_orb);
  c.partial = off; off = al256(off + 2 * sizeof(double) * (size_t)(d.n_items > 0 ? d.n_items : 1));
  c.e_trip = off;  off = al256(off + sizeof(double) * (size_t)(d.n_trip > 0 ? d.n_trip : 1));
  c.out = off;     off = al256(off + 4 * sizeof(double));
  c.counter = off; off = al256(off + 2 * sizeof(unsigned));
  c.total = off;
  return c;
}

// Work decomposition of the FP64 kernel with as many orbits per item as it
// takes for the scratch to fit the static array.
bool plan(int o, int v, tc::Dims *out, Carve *cv) {
  tc::Dims d{};
  d.o = o;
  d.v = v;
  d.nt = tc::fp64_tile();
  d.ntiles = (v + d.nt - 1) / d.nt;
  const long long T = d.ntiles;
  d.n_trip = (int)((long long)o * (o + 1) * (o + 2) / 6 - o);
  const long long n_orb = T * (T + 1) * (T + 2) / 6;
  if (n_orb > (1LL << 30)) return false;
  d.n_orb = (int)n_orb;
  for (long long opi = 1;; opi *= 2) {
    if (opi > n_orb) opi = n_orb;
    d.orb_per_item = (int)opi;
    d.items_per_trip = (int)((n_orb + opi - 1) / opi);
    d.n_items = (long long)d.n_trip * d.items_per_trip;
    const Carve c = carve(d);
    if (c.total <= kScratchBytes) { *out = d; *cv = c; return true; }
    if (opi == n_orb) return false;
  }
}

// Work tables written on the device: triplets i >= j >= k (all-equal ones
// dropped) and tile orbits P >= Q >= R, each at its position in the
// lexicographic enumeration the fused kernel expects.
__global__ void fill_tables(int o, int ntiles, int4 *trip, int4 *orb) {
  const long long no3 = (long long)o * o * o;
  const long long nt3 = (long long)ntiles * ntiles * ntiles;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < no3 + nt3;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < no3) {
      const int i = (int)(e / ((long long)o * o)), j = (int)((e / o) % o), k = (int)(e % o);
      if (i >= j && j >= k && i != k) {
        const long long pos = (long long)i * (i + 1) * (i + 2) / 6 + (long long)j * (j + 1) / 2 + k - i;
        trip[pos] = make_int4(i, j, k, 2 - (i == j) - (j == k));
      }
    } else {
      const long long f = e - no3;
      const int P = (int)(f / ((long long)ntiles * ntiles)), Q = (int)((f / ntiles) % ntiles), R = (int)(f % ntiles);
      if (P >= Q && Q >= R) {
        const long long pos = (long long)P * (P + 1) * (P + 2) / 6 + (long long)Q * (Q + 1) / 2 + R;
        orb[pos] = make_int4(P, Q, R, 0);
      }
    }
  }
}

tc_status err(char *buf, size_t len, tc_status s, const char *msg, const char *detail = nullptr) {
  if (buf && len > 0) snprintf(buf, len, "%s%s%s", msg, detail ? ": " : "", detail ? detail : "");
  return s;
}

}  // namespace

extern "C" tc_status tc_energy_dev_noalloc(int o, int v, const double *eps, const double *t1, const double *t2,
                                           const tc_ints *ints, double *e_t_dev, double *e_ijk_dev, void *stream,
                                           char *errbuf, size_t errlen) {
  if (errbuf && errlen > 0) errbuf[0] = '\0';
  if (o <= 0 || v <= 0) return err(errbuf, errlen, TC_EINVAL, "o and v must be positive");
  if (!eps || !t1 || !t2 || !ints || !ints->ovvv || !ints->ovoo || !ints->ovov || !e_t_dev)
    return err(errbuf, errlen, TC_EINVAL, "NULL input or output array");
  tc::Dims d{};
  Carve cv{};
  if (!plan(o, v, &d, &cv))
    return err(errbuf, errlen, TC_ENOMEM,
               "job too large for the static scratch array (TC_NOALLOC_SCRATCH_BYTES); use tc_energy_dev");

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return err(errbuf, errlen, TC_ECUDA, "cudaGetDevice", cudaGetErrorString(ce));
  if (dev < 0 || dev >= kMaxDevices) return err(errbuf, errlen, TC_EINVAL, "device ordinal out of range");
  DeviceSetup su;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.ready) {                          // once per device, with that device current
      void *p = nullptr;
      ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (ce != cudaSuccess) return err(errbuf, errlen, TC_ECUDA, "cudaGetSymbolAddress", cudaGetErrorString(ce));
      ce = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
      if (ce != cudaSuccess) return err(errbuf, errlen, TC_ECUDA, "cudaDeviceGetAttribute", cudaGetErrorString(ce));
      ce = tc::fp64_blocks_per_sm(&s.blocks_per_sm);
      if (ce != cudaSuccess) return err(errbuf, errlen, TC_ECUDA, "kernel set-up", cudaGetErrorString(ce));
      s.scratch = (unsigned char *)p;
      s.ready = true;
    }
    su = s;
  }

  cudaStream_t st = (cudaStream_t)stream;
  unsigned char *base = su.scratch;
  tc::Work w{};
  int4 *trip = (int4 *)(base + cv.trip);
  int4 *orb = (int4 *)(base + cv.orb);
  w.trip = trip;
  w.orb = orb;
  w.partial = (double *)(base + cv.partial);
  w.counter = (unsigned *)(base + cv.counter);
  w.err = (int *)(base + cv.counter + sizeof(unsigned));
  double *e_trip = (double *)(base + cv.e_trip);
  double *out = (double *)(base + cv.out);
  tc::Inputs in{eps, t1, t2, ints->ovvv, ints->ovoo, ints->ovov};

#define NA_CUDA(call)                                                                    \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return err(errbuf, errlen, TC_ECUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

  NA_CUDA(cudaMemsetAsync(w.counter, 0, 2 * sizeof(unsigned), st));
  if (e_ijk_dev) NA_CUDA(cudaMemsetAsync(e_ijk_dev, 0, sizeof(double) * (size_t)o * o * o, st));
  const long long nfill = (long long)o * o * o + (long long)d.ntiles * d.ntiles * d.ntiles;
  const int fill_blocks = (int)((nfill + 255) / 256 < 4096 ? (nfill + 255) / 256 : 4096);
  fill_tables<<<fill_blocks, 256, 0, st>>>(o, d.ntiles, trip, orb);
  NA_CUDA(cudaGetLastError());
  if (d.n_items > 0) {
    long long grid = (long long)su.num_sms * su.blocks_per_sm;
    if (grid > d.n_items) grid = d.n_items;
    tc::FpBatch b{};
    b.njobs = 1;
    b.total_items = d.n_items;
    b.counter = w.counter;
    b.job[0] = tc::FpJob{d, in, w, 0};
    NA_CUDA(tc::launch_fp64(b, (int)grid, st));
  }
  {
    tc::RedBatch rb{};
    rb.njobs = 1;
    rb.job[0] = tc::RedJob{d.n_trip, d.items_per_trip, o, w.trip, w.partial, e_trip, e_ijk_dev, out};
    NA_CUDA(tc::launch_reduce(rb, st));
  }
  NA_CUDA(cudaMemcpyAsync(e_t_dev, out, sizeof(double), cudaMemcpyDeviceToDevice, st));
#undef NA_CUDA
  return TC_OK;
}
