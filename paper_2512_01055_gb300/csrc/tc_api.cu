// C ABI of the (T) library (include/tc.h): argument checks, HBM admission,
// device workspace reuse, work tables, launches and the final read-back of
// the blocking entry points, and the assembly of the integrals from
// density-fitting factors (Eq. 6) for tc_energy_df_dev.  The serving entry
// points are in tc_serve.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/tc.h"
#include "tc_ctx.h"
#include "tc_internal.cuh"
#include "tc_plan.cuh"

namespace {

tc_status fail(tc_ctx *ctx, tc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return s;
}

#define TC_CUDA(ctx, call)                                                                  \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, TC_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                      \
  } while (0)

tc_status check_args(tc_ctx *ctx, int o, int v, const double *eps, const double *t1, const double *t2,
                     const tc_ints *ints, int *prec, int *slices) {
  if (!ctx) return TC_EINVAL;
  if (o <= 0 || v <= 0) return fail(ctx, TC_EINVAL, "o and v must be positive (o=%d v=%d)", o, v);
  if ((long long)o * v * v * v > (1LL << 40)) return fail(ctx, TC_EINVAL, "o*v^3 too large");
  if (!eps || !t1 || !t2 || !ints || !ints->ovvv || !ints->ovoo || !ints->ovov)
    return fail(ctx, TC_EINVAL, "NULL input array");
  if (*prec < 0) *prec = ctx->default_prec;
  if (*prec != TC_FP64 && *prec != TC_SPLIT_BF16) return fail(ctx, TC_EINVAL, "unknown precision %d", *prec);
  if (*prec == TC_SPLIT_BF16) {
    if (*slices <= 0) *slices = ctx->default_slices;
    if (*slices < 2 || *slices > 4) return fail(ctx, TC_EINVAL, "slices must be 2, 3 or 4 (got %d)", *slices);
  } else {
    *slices = 0;
  }
  return TC_OK;
}

double alg_flops(int o, int v) {
  const double O = o, V = v;
  return 2.0 * (O * O * O * V * V * V * V + O * O * O * O * V * V * V);
}

// Inputs that are still arriving (tc_energy, split path): chunk c holds the
// rows of t2, ovvv, ovoo and ovov whose first occupied index lies in
// [c ? p_end[c - 1] : 0, p_end[c]); ready[c] is recorded once they are on the
// device.  Triplets run in the order i >= j >= k with i non-decreasing, and a
// triplet reads only rows p <= i, so a block of triplets needs the chunks up
// to the one holding its last triplet's i.
struct Staging {
  int nchunk = 0;
  const int *p_end = nullptr;
  const cudaEvent_t *ready = nullptr;
};

// The hot path on device-resident inputs.  Caller holds ctx->mu.
// subset (optional): process these triplets only; e_sub receives their sums.
// stg (optional, split path, no subset): slice each chunk of the inputs once
// it has arrived, just before the first block of triplets that reads it.
tc_status run_device(tc_ctx *ctx, int o, int v, const tc::Inputs &in, int prec, int slices, double *e_ijk_dev,
                     cudaStream_t st, tc_result *out, const std::vector<int4> *subset = nullptr,
                     std::vector<double> *e_sub = nullptr, const Staging *stg = nullptr) {
  const bool split = (prec == TC_SPLIT_BF16);
  const int nt = split ? tc::split_tile() : tc::fp64_tile();
  const tc::Dims d = tc::plan::make_dims(o, v, nt, subset ? (int)subset->size() : -1,
                                         split ? tc::split_orb_per_item(o, v, slices) : 1);
  const tc::plan::Layout L = tc::plan::make_layout(d);
  const tc::SplitLayout SL = split ? tc::split_layout(o, v, slices) : tc::SplitLayout{};
  const size_t need = L.total + SL.total;
  if (need > ctx->budget) return fail(ctx, TC_ENOMEM, "workspace %zu B exceeds budget %zu B", need, ctx->budget);
  TC_CUDA(ctx, ctx->ws.ensure(L.total));
  if (split) TC_CUDA(ctx, ctx->ws_split.ensure(SL.total));
  char *base = (char *)ctx->ws.p;
  const std::vector<int4> tab = tc::plan::tables(d, L, subset);
  TC_CUDA(ctx, cudaMemcpyAsync(base + L.trip, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  tc::Work w{};
  w.trip = (const int4 *)(base + L.trip);
  w.orb = (const int4 *)(base + L.orb);
  w.partial = (double *)(base + L.partial);
  w.counter = (unsigned *)(base + L.counter);
  w.err = (int *)(base + L.counter + sizeof(unsigned));
  double *e_trip = (double *)(base + L.e_trip);
  double *dout = (double *)(base + L.out);
  TC_CUDA(ctx, cudaMemsetAsync(w.counter, 0, 2 * sizeof(unsigned), st));
  if (e_ijk_dev) TC_CUDA(ctx, cudaMemsetAsync(e_ijk_dev, 0, sizeof(double) * (size_t)o * o * o, st));
  int launches = 1;                                      // reduce_jobs
  int nblocks = 0;                                       // split path: blocks of triplets
  if (stg && (!split || subset)) return fail(ctx, TC_EINTERNAL, "staged inputs need the split path on all triplets");
  int staged = 0;                                        // chunks sliced so far
  const int npev = stg ? 2 * (stg->nchunk + 1) : 0;
  while ((int)ctx->pev.size() < npev) {
    cudaEvent_t e = nullptr;
    TC_CUDA(ctx, cudaEventCreate(&e));
    ctx->pev.push_back(e);
  }
  // wait for and slice every chunk that starts at or below first index imax
  auto stage_upto = [&](int imax) -> tc_status {
    for (; staged < stg->nchunk && (staged ? stg->p_end[staged - 1] : 0) <= imax; ++staged) {
      const int p0 = staged ? stg->p_end[staged - 1] : 0, p1 = stg->p_end[staged];
      TC_CUDA(ctx, cudaStreamWaitEvent(st, stg->ready[staged], 0));
      TC_CUDA(ctx, cudaEventRecord(ctx->pev[2 + 2 * staged], st));
      TC_CUDA(ctx, tc::launch_split_prep_range(SL, in, ctx->ws_split.p, st, p0, p1));
      TC_CUDA(ctx, cudaEventRecord(ctx->pev[3 + 2 * staged], st));
      launches += tc::split_prep_range_launches();
    }
    return TC_OK;
  };
  if (split && stg) {
    TC_CUDA(ctx, cudaEventRecord(ctx->pev[0], st));
    TC_CUDA(ctx, tc::launch_split_prep_common(SL, in, ctx->ws_split.p, st));
    TC_CUDA(ctx, cudaEventRecord(ctx->pev[1], st));
    launches += tc::split_prep_launches() - tc::split_prep_range_launches();
  } else if (split) {
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[2], st));
    TC_CUDA(ctx, tc::launch_split_prep(SL, in, ctx->ws_split.p, st));
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[3], st));
    launches += tc::split_prep_launches();
  }
  if (d.n_items > 0) {
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[0], st));
    if (split) {
      // blocks of nb triplets: the three W-term GEMM launches sum W into the
      // W buffer, then the energy launch runs over the block's orbits
      const int nb = SL.g.nb;
      nblocks = (d.n_trip + nb - 1) / nb;
      while ((int)ctx->wev.size() < 2 * nblocks) {
        cudaEvent_t e = nullptr;
        TC_CUDA(ctx, cudaEventCreate(&e));
        ctx->wev.push_back(e);
      }
      static thread_local tc::WtBatch wb;
      static thread_local tc::EnBatch eb;
      for (int blk = 0; blk < nblocks; ++blk) {
        const int t0 = blk * nb, nt = std::min(nb, d.n_trip - t0);
        if (stg) {
          const tc_status ss = stage_upto(tab[(size_t)t0 + nt - 1].x);
          if (ss != TC_OK) return ss;
        }
        wb = tc::WtBatch{};
        wb.njobs = 1;
        wb.err = w.err;
        wb.job[0] = tc::wt_job(SL, ctx->ws_split.p, w.trip, t0, nt);
        eb = tc::EnBatch{};
        eb.njobs = 1;
        eb.err = w.err;
        TC_CUDA(ctx, tc::en_job(&eb.job[0], d, SL, ctx->ws_split.p, in, w, t0, nt));
        TC_CUDA(ctx, tc::launch_split_block(wb, eb, slices, ctx->num_sms, st, ctx->wev[2 * blk], ctx->wev[2 * blk + 1]));
      }
      launches += (tc::SPLIT_WT_LAUNCHES + 1) * nblocks - 1;
    } else {
      int per_sm = 0;
      TC_CUDA(ctx, tc::fp64_blocks_per_sm(&per_sm));
      long long grid = (long long)ctx->num_sms * per_sm;
      grid = std::min<long long>(grid, d.n_items);
      tc::FpBatch b{};
      b.njobs = 1;
      b.total_items = d.n_items;
      b.counter = w.counter;
      b.job[0] = tc::FpJob{d, in, w, 0, 0};
      TC_CUDA(ctx, tc::launch_fp64(b, (int)grid, st));
    }
    TC_CUDA(ctx, cudaEventRecord(ctx->ev[1], st));
    launches += 1;
  }
  if (stg) {
    // the remaining chunks (read by no triplet, e.g. o = 1): the stream still
    // waits for their copies before the read-back
    const tc_status ss = stage_upto(o);
    if (ss != TC_OK) return ss;
  }
  {
    tc::RedBatch rb{};
    rb.njobs = 1;
    rb.job[0] = tc::RedJob{d.n_trip, d.items_per_trip, o, w.trip, w.partial, e_trip, e_ijk_dev, dout};
    TC_CUDA(ctx, tc::launch_reduce(rb, st));
  }
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->host_out, dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->host_out + 3, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TC_CUDA(ctx, cudaStreamSynchronize(st));
  int errflag = 0;
  std::memcpy(&errflag, ctx->host_out + 3, sizeof(int));
  if (errflag != 0)
    return fail(ctx, (errflag >= 11 && errflag <= 15) ? TC_ETIMEOUT : TC_EINTERNAL,
                "device-side wait gave up (code %d)", errflag);
  out->e_t = ctx->host_out[0];
  out->e_t5 = ctx->host_out[2];
  if (e_sub) {
    e_sub->assign((size_t)d.n_trip, 0.0);
    if (d.n_trip > 0) {
      TC_CUDA(ctx, cudaMemcpyAsync(e_sub->data(), e_trip, sizeof(double) * (size_t)d.n_trip, cudaMemcpyDeviceToHost, st));
      TC_CUDA(ctx, cudaStreamSynchronize(st));
    }
  }
  if (d.n_items > 0) {
    float ms = 0.f;
    TC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
    out->kernel_seconds = 1e-3 * ms;
    out->wterm_seconds = out->kernel_seconds;
    if (split) {
      double wsum = 0.0;
      for (int blk = 0; blk < nblocks; ++blk) {
        TC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->wev[2 * blk], ctx->wev[2 * blk + 1]));
        wsum += 1e-3 * ms;
      }
      out->wterm_seconds = wsum;
    }
  }
  if (split && stg) {
    double psum = 0.0;
    for (int c = 0; c <= stg->nchunk; ++c) {
      float ms = 0.f;
      TC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->pev[2 * c], ctx->pev[2 * c + 1]));
      psum += 1e-3 * ms;
    }
    out->prep_seconds = psum;
  } else if (split) {
    float ms = 0.f;
    TC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
    out->prep_seconds = 1e-3 * ms;
  }
  out->n_items = d.n_items;
  out->launches = launches;
  out->prec = prec;
  out->slices = (prec == TC_FP64) ? 0 : slices;
  out->o = o;
  out->v = v;
  return TC_OK;
}

// Device bytes tc_energy_df(_dev) holds besides the workspace: the assembled
// integrals and the assembly's scratch (scales and digit images of B).
size_t df_bytes(int o, int v, int nq) {
  const size_t n_ovvv = (size_t)o * v * v * v, n_ovoo = (size_t)o * v * o * o, n_ovov = (size_t)o * v * o * v;
  return sizeof(double) * (n_ovvv + n_ovoo + n_ovov) + tc::df_scratch_bytes(o, v, nq);
}

// The integrals from the DF factors B (device) on st, then the energy (Eq. 6,
// then the path of tc_energy_dev).  Caller holds ctx->mu and checked the
// arguments and the budget.
tc_status df_energy(tc_ctx *ctx, int o, int v, int nq, const double *eps, const double *t1, const double *t2,
                    const double *B, int prec, int slices, double *e_ijk_dev, cudaStream_t st, tc_result *out) {
  const size_t n_ovvv = (size_t)o * v * v * v, n_ovoo = (size_t)o * v * o * o, n_ovov = (size_t)o * v * o * v;
  TC_CUDA(ctx, ctx->in_ovvv.ensure(sizeof(double) * n_ovvv));
  TC_CUDA(ctx, ctx->in_ovoo.ensure(sizeof(double) * n_ovoo));
  TC_CUDA(ctx, ctx->in_ovov.ensure(sizeof(double) * n_ovov));
  TC_CUDA(ctx, ctx->df_b.ensure(tc::df_scratch_bytes(o, v, nq)));
  for (auto &e : ctx->dfev)
    if (!e) TC_CUDA(ctx, cudaEventCreate(&e));
  double *ovvv = (double *)ctx->in_ovvv.p, *ovoo = (double *)ctx->in_ovoo.p, *ovov = (double *)ctx->in_ovov.p;
  TC_CUDA(ctx, cudaEventRecord(ctx->dfev[0], st));
  int digits = 0;
  TC_CUDA(ctx, tc::df_assemble(B, nq, o, v, ovvv, ovoo, ovov, ctx->df_b.p, ctx->num_sms, st, &digits));
  TC_CUDA(ctx, cudaEventRecord(ctx->dfev[1], st));
  const tc::Inputs in{eps, t1, t2, ovvv, ovoo, ovov};
  const tc_status s = run_device(ctx, o, v, in, prec, slices, e_ijk_dev, st, out);
  if (s != TC_OK) return s;
  int derr = 0;
  TC_CUDA(ctx, cudaMemcpy(&derr, tc::df_error_flag(ctx->df_b.p, o, v, nq), sizeof(int), cudaMemcpyDeviceToHost));
  if (derr != 0) return fail(ctx, TC_ETIMEOUT, "integral assembly: device-side wait gave up (code %d)", derr);
  float ms = 0.f;
  TC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->dfev[0], ctx->dfev[1]));
  out->df_seconds = 1e-3 * ms;
  out->df_digits = digits;
  return TC_OK;
}

}  // namespace

extern "C" {

const char *tc_status_str(tc_status s) {
  switch (s) {
    case TC_OK: return "TC_OK";
    case TC_EINVAL: return "TC_EINVAL";
    case TC_ENOMEM: return "TC_ENOMEM";
    case TC_ECUDA: return "TC_ECUDA";
    case TC_ENOTREADY: return "TC_ENOTREADY";
    case TC_ETIMEOUT: return "TC_ETIMEOUT";
    case TC_EBUSY: return "TC_EBUSY";
    case TC_ECANCELLED: return "TC_ECANCELLED";
    case TC_EINTERNAL: return "TC_EINTERNAL";
  }
  return "TC_UNKNOWN";
}

const char *tc_last_error(tc_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

size_t tc_workspace_bytes(int o, int v, int prec, int slices) {
  if (o <= 0 || v <= 0) return 0;
  const bool split = (prec == TC_SPLIT_BF16);
  if (split && slices <= 0) slices = 3;
  const tc::Dims d = split ? tc::plan::make_dims(o, v, tc::split_tile(), -1, tc::split_orb_per_item(o, v, slices))
                           : tc::plan::make_dims(o, v, tc::fp64_tile());
  return tc::plan::make_layout(d).total + (split ? tc::split_layout(o, v, slices).total : 0);
}

tc_status tc_init(tc_ctx **out, const tc_options *opt) {
  if (!out) return TC_EINVAL;
  *out = nullptr;
  tc_ctx *ctx = new (std::nothrow) tc_ctx();
  if (!ctx) return TC_ENOMEM;
  if (opt) {
    ctx->device = opt->device;
    ctx->budget = opt->hbm_budget_bytes;
    ctx->default_prec = opt->default_prec;
    ctx->default_slices = opt->default_slices > 0 ? opt->default_slices : 3;
    ctx->timeout_ms = opt->timeout_ms > 0 ? opt->timeout_ms : 60000;
    if (opt->max_inflight > 0) ctx->max_inflight = std::min(opt->max_inflight, tc::MAX_BATCH);
    if (opt->max_queue > 0) ctx->max_queue = opt->max_queue;
    if (opt->iteration_ms > 0) ctx->iteration_ms = opt->iteration_ms;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ctx->device < 0 || ctx->device >= ndev) {
    delete ctx;
    return TC_ECUDA;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void **)&ctx->host_out, 4 * sizeof(double)) != cudaSuccess ||
      cudaEventCreate(&ctx->ev[0]) != cudaSuccess || cudaEventCreate(&ctx->ev[1]) != cudaSuccess ||
      cudaEventCreate(&ctx->ev[2]) != cudaSuccess || cudaEventCreate(&ctx->ev[3]) != cudaSuccess) {
    delete ctx;
    return TC_ECUDA;
  }
  if (ctx->budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = (size_t)(0.9 * (double)fr);
  }
  *out = ctx;
  return TC_OK;
}

void tc_finalize(tc_ctx *ctx) {
  if (!ctx) return;
  if (ctx->server) tc::server_destroy(ctx->server);   // stops the scheduler, releases its jobs
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->ws.release();
  ctx->ws_split.release();
  ctx->in_eps.release(); ctx->in_t1.release(); ctx->in_t2.release();
  ctx->in_ovvv.release(); ctx->in_ovoo.release(); ctx->in_ovov.release();
  ctx->df_b.release();
  ctx->df_in.release();
  for (auto &e : ctx->dfev) if (e) cudaEventDestroy(e);
  if (ctx->host_out) cudaFreeHost(ctx->host_out);
  for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
  for (auto &e : ctx->wev) if (e) cudaEventDestroy(e);
  for (auto &e : ctx->cev) if (e) cudaEventDestroy(e);
  for (auto &e : ctx->pev) if (e) cudaEventDestroy(e);
  if (ctx->copy_stream) {
    cudaStreamSynchronize(ctx->copy_stream);
    cudaStreamDestroy(ctx->copy_stream);
  }
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

tc_status tc_energy_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1, const double *t2,
                        const tc_ints *ints, int prec, int slices, double *e_ijk_dev, void *stream,
                        tc_result *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  tc_status s = check_args(ctx, o, v, eps, t1, t2, ints, &prec, &slices);
  if (s != TC_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  tc::Inputs in{eps, t1, t2, ints->ovvv, ints->ovoo, ints->ovov};
  std::memset(out, 0, sizeof *out);
  s = run_device(ctx, o, v, in, prec, slices, e_ijk_dev, (cudaStream_t)stream, out);
  if (s != TC_OK) return s;
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out->tflops_alg = alg_flops(o, v) / std::max(out->seconds, 1e-12) / 1e12;
  return TC_OK;
}

tc_status tc_energy_df_dev(tc_ctx *ctx, int o, int v, int nq, const double *eps, const double *t1,
                           const double *t2, const double *B, int prec, int slices, double *e_ijk_dev, void *stream,
                           tc_result *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  if (nq <= 0 || !B) return fail(ctx, TC_EINVAL, "nq must be positive and B non-NULL (nq=%d)", nq);
  const tc_ints probe{B, B, B};                       // the integrals are formed from B
  tc_status s = check_args(ctx, o, v, eps, t1, t2, &probe, &prec, &slices);
  if (s != TC_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  if (df_bytes(o, v, nq) + tc_workspace_bytes(o, v, prec, slices) > ctx->budget)
    return fail(ctx, TC_ENOMEM, "job needs %zu B, budget %zu B", df_bytes(o, v, nq) + tc_workspace_bytes(o, v, prec, slices),
                ctx->budget);
  std::memset(out, 0, sizeof *out);
  s = df_energy(ctx, o, v, nq, eps, t1, t2, B, prec, slices, e_ijk_dev, (cudaStream_t)stream, out);
  if (s != TC_OK) return s;
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out->tflops_alg = alg_flops(o, v) / std::max(out->seconds, 1e-12) / 1e12;
  return TC_OK;
}

tc_status tc_energy_df(tc_ctx *ctx, int o, int v, int nq, const double *eps, const double *t1, const double *t2,
                       const double *B, int prec, int slices, double *e_ijk, tc_result *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  if (nq <= 0 || !B) return fail(ctx, TC_EINVAL, "nq must be positive and B non-NULL (nq=%d)", nq);
  const tc_ints probe{B, B, B};
  tc_status s = check_args(ctx, o, v, eps, t1, t2, &probe, &prec, &slices);
  if (s != TC_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t n_eps = (size_t)o + v, n_t1 = (size_t)o * v, n_t2 = (size_t)o * o * v * v;
  const size_t n_b = (size_t)nq * (o + v) * (o + v);
  const size_t in_bytes = sizeof(double) * (n_eps + (size_t)o * o * o + n_t1 + n_t2 + n_b);
  const size_t need = in_bytes + df_bytes(o, v, nq) + tc_workspace_bytes(o, v, prec, slices);
  if (need > ctx->budget) return fail(ctx, TC_ENOMEM, "job needs %zu B, budget %zu B", need, ctx->budget);
  cudaStream_t st = ctx->stream;
  TC_CUDA(ctx, ctx->in_eps.ensure(sizeof(double) * (n_eps + (size_t)o * o * o)));
  TC_CUDA(ctx, ctx->in_t1.ensure(sizeof(double) * n_t1));
  TC_CUDA(ctx, ctx->in_t2.ensure(sizeof(double) * n_t2));
  TC_CUDA(ctx, ctx->df_in.ensure(sizeof(double) * n_b));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_eps.p, eps, sizeof(double) * n_eps, cudaMemcpyHostToDevice, st));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_t1.p, t1, sizeof(double) * n_t1, cudaMemcpyHostToDevice, st));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_t2.p, t2, sizeof(double) * n_t2, cudaMemcpyHostToDevice, st));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->df_in.p, B, sizeof(double) * n_b, cudaMemcpyHostToDevice, st));
  double *e_ijk_dev = e_ijk ? (double *)ctx->in_eps.p + n_eps : nullptr;
  std::memset(out, 0, sizeof *out);
  s = df_energy(ctx, o, v, nq, (const double *)ctx->in_eps.p, (const double *)ctx->in_t1.p,
                (const double *)ctx->in_t2.p, (const double *)ctx->df_in.p, prec, slices, e_ijk_dev, st, out);
  if (s != TC_OK) return s;
  if (e_ijk) {
    TC_CUDA(ctx, cudaMemcpyAsync(e_ijk, e_ijk_dev, sizeof(double) * (size_t)o * o * o, cudaMemcpyDeviceToHost, st));
    TC_CUDA(ctx, cudaStreamSynchronize(st));
  }
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out->tflops_alg = alg_flops(o, v) / std::max(out->seconds, 1e-12) / 1e12;
  return TC_OK;
}

tc_status tc_triplets_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1, const double *t2,
                          const tc_ints *ints, int prec, int slices, const int *trip, int n, double *e_out,
                          void *stream, tc_result *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  tc_status s = check_args(ctx, o, v, eps, t1, t2, ints, &prec, &slices);
  if (s != TC_OK) return s;
  if (n < 0 || (n > 0 && (!trip || !e_out))) return fail(ctx, TC_EINVAL, "bad triplet list");
  std::vector<int4> sub;
  std::vector<int> where;                  // position in the caller's list of each processed triplet
  for (int m = 0; m < n; ++m) {
    const int i = trip[3 * m], j = trip[3 * m + 1], k = trip[3 * m + 2];
    if (!(o > i && i >= j && j >= k && k >= 0))
      return fail(ctx, TC_EINVAL, "triplet %d = (%d, %d, %d) is not o > i >= j >= k >= 0", m, i, j, k);
  }
  for (int m = 0; m < n; ++m) {
    const int i = trip[3 * m], j = trip[3 * m + 1], k = trip[3 * m + 2];
    e_out[m] = 0.0;
    if (i == k) continue;
    sub.push_back(make_int4(i, j, k, 2 - (i == j) - (j == k)));
    where.push_back(m);
  }
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  tc::Inputs in{eps, t1, t2, ints->ovvv, ints->ovoo, ints->ovov};
  std::memset(out, 0, sizeof *out);
  std::vector<double> e_sub;
  s = run_device(ctx, o, v, in, prec, slices, nullptr, (cudaStream_t)stream, out, &sub, &e_sub);
  if (s != TC_OK) return s;
  for (size_t q = 0; q < where.size(); ++q) e_out[where[q]] = e_sub[q];
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return TC_OK;
}

// ---------------------------------------------------------------- one energy over several ranks

tc_status tc_shard_range(int o, int rank, int world, long long *first, long long *count) {
  if (o <= 0 || world <= 0 || rank < 0 || rank >= world || !first || !count) return TC_EINVAL;
  const long long n = (long long)o * (o + 1) * (o + 2) / 6 - o;   // i >= j >= k, all-equal ones excluded
  const long long a = n * rank / world, b = n * (rank + 1) / world;
  *first = a;
  *count = b - a;
  return TC_OK;
}

tc_status tc_sum_parts(const double *x, long long n, double *part) {
  if (n < 0 || (n > 0 && !x) || !part) return TC_EINVAL;
  double s = 0.0, c = 0.0;
  for (long long m = 0; m < n; ++m) {                 // Neumaier's compensated sum, in order
    const double t = s + x[m];
    c += (std::fabs(s) >= std::fabs(x[m])) ? ((s - t) + x[m]) : ((x[m] - t) + s);
    s = t;
  }
  part[0] = s;
  part[1] = c;
  return TC_OK;
}

tc_status tc_combine_parts(const double *parts, int n, double *e_t) {
  if (n < 0 || (n > 0 && !parts) || !e_t) return TC_EINVAL;
  double s = 0.0, c = 0.0, cc = 0.0;
  for (int r = 0; r < n; ++r) {                       // rank order: the same bits on every rank
    const double x = parts[2 * r];
    const double t = s + x;
    c += (std::fabs(s) >= std::fabs(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
    cc += parts[2 * r + 1];
  }
  *e_t = s + (c + cc);
  return TC_OK;
}

tc_status tc_energy_shard_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1, const double *t2,
                              const tc_ints *ints, int prec, int slices, int rank, int world, double *part,
                              void *stream, tc_result *out) {
  if (!ctx || !out || !part) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  tc_status s = check_args(ctx, o, v, eps, t1, t2, ints, &prec, &slices);
  if (s != TC_OK) return s;
  long long first = 0, count = 0;
  if (tc_shard_range(o, rank, world, &first, &count) != TC_OK)
    return fail(ctx, TC_EINVAL, "rank %d of world %d is not a valid shard", rank, world);
  // the rank's contiguous range of the triplet order (i, j, k) lexicographic
  std::vector<int4> sub;
  sub.reserve((size_t)count);
  long long idx = 0;
  for (int i = 0; i < o && idx < first + count; ++i)
    for (int j = 0; j <= i && idx < first + count; ++j)
      for (int k = 0; k <= j && idx < first + count; ++k) {
        if (i == k) continue;
        if (idx >= first) sub.push_back(make_int4(i, j, k, 2 - (i == j) - (j == k)));
        ++idx;
      }
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  tc::Inputs in{eps, t1, t2, ints->ovvv, ints->ovoo, ints->ovov};
  std::memset(out, 0, sizeof *out);
  std::vector<double> e_sub;
  if (!sub.empty()) {
    s = run_device(ctx, o, v, in, prec, slices, nullptr, (cudaStream_t)stream, out, &sub, &e_sub);
    if (s != TC_OK) return s;
  }
  tc_sum_parts(e_sub.data(), (long long)e_sub.size(), part);
  out->e_t = part[0] + part[1];
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return TC_OK;
}

tc_status tc_energy(tc_ctx *ctx, int o, int v, const double *eps, const double *t1, const double *t2,
                    const tc_ints *ints, int prec, int slices, double *e_ijk, tc_result *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->err.clear();
  tc_status s = check_args(ctx, o, v, eps, t1, t2, ints, &prec, &slices);
  if (s != TC_OK) return s;
  const auto t0 = std::chrono::steady_clock::now();
  TC_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t n_eps = (size_t)o + v, n_t1 = (size_t)o * v, n_t2 = (size_t)o * o * v * v;
  const size_t n_ovvv = (size_t)o * v * v * v, n_ovoo = (size_t)o * v * o * o, n_ovov = (size_t)o * v * o * v;
  const size_t in_bytes = sizeof(double) * (n_eps + n_t1 + n_t2 + n_ovvv + n_ovoo + n_ovov + (size_t)o * o * o);
  if (in_bytes + tc_workspace_bytes(o, v, prec, slices) > ctx->budget)
    return fail(ctx, TC_ENOMEM, "job needs %zu B, budget %zu B", in_bytes + tc_workspace_bytes(o, v, prec, slices),
                ctx->budget);
  cudaStream_t st = ctx->stream;
  TC_CUDA(ctx, ctx->in_eps.ensure(sizeof(double) * (n_eps + (size_t)o * o * o)));
  TC_CUDA(ctx, ctx->in_t1.ensure(sizeof(double) * n_t1));
  TC_CUDA(ctx, ctx->in_t2.ensure(sizeof(double) * n_t2));
  TC_CUDA(ctx, ctx->in_ovvv.ensure(sizeof(double) * n_ovvv));
  TC_CUDA(ctx, ctx->in_ovoo.ensure(sizeof(double) * n_ovoo));
  TC_CUDA(ctx, ctx->in_ovov.ensure(sizeof(double) * n_ovov));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_eps.p, eps, sizeof(double) * n_eps, cudaMemcpyHostToDevice, st));
  TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_t1.p, t1, sizeof(double) * n_t1, cudaMemcpyHostToDevice, st));
  tc::Inputs in{(const double *)ctx->in_eps.p, (const double *)ctx->in_t1.p, (const double *)ctx->in_t2.p,
                (const double *)ctx->in_ovvv.p, (const double *)ctx->in_ovoo.p, (const double *)ctx->in_ovov.p};
  double *e_ijk_dev = e_ijk ? (double *)ctx->in_eps.p + n_eps : nullptr;
  std::memset(out, 0, sizeof *out);
  if (prec == TC_SPLIT_BF16) {
    // The four large inputs go over on the copy stream in chunks of occupied
    // indices (their first index), and each chunk is sliced just before the
    // first block of triplets that reads it, so the copies of the later
    // chunks overlap the first blocks' tensor-core work.  At most 64 chunks.
    const int per = std::max(1, (o + 63) / 64), nchunk = (o + per - 1) / per;
    std::vector<int> p_end((size_t)nchunk);
    for (int c = 0; c < nchunk; ++c) p_end[(size_t)c] = std::min(o, (c + 1) * per);
    while ((int)ctx->cev.size() < nchunk) {
      cudaEvent_t e = nullptr;
      TC_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ctx->cev.push_back(e);
    }
    const struct { void *dst; const double *src; size_t row; } big[4] = {
        {ctx->in_t2.p, t2, (size_t)o * v * v},
        {ctx->in_ovvv.p, ints->ovvv, (size_t)v * v * v},
        {ctx->in_ovoo.p, ints->ovoo, (size_t)v * o * o},
        {ctx->in_ovov.p, ints->ovov, (size_t)v * o * v}};
    cudaError_t ce = cudaSuccess;
    for (int c = 0; c < nchunk && ce == cudaSuccess; ++c) {
      const size_t p0 = c ? (size_t)p_end[(size_t)c - 1] : 0, np = (size_t)p_end[(size_t)c] - p0;
      for (int k = 0; k < 4 && ce == cudaSuccess; ++k)
        ce = cudaMemcpyAsync((double *)big[k].dst + p0 * big[k].row, big[k].src + p0 * big[k].row,
                             sizeof(double) * np * big[k].row, cudaMemcpyHostToDevice, ctx->copy_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(ctx->cev[(size_t)c], ctx->copy_stream);
    }
    if (ce == cudaSuccess) {
      const Staging stg{nchunk, p_end.data(), ctx->cev.data()};
      s = run_device(ctx, o, v, in, prec, slices, e_ijk_dev, st, out, nullptr, nullptr, &stg);
    }
    // no copy may still read the caller's arrays once this call returns
    const cudaError_t ce2 = cudaStreamSynchronize(ctx->copy_stream);
    if (ce == cudaSuccess) ce = ce2;
    if (ce != cudaSuccess)
      return fail(ctx, TC_ECUDA, "input copies failed: %s", cudaGetErrorString(ce));
  } else {
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_t2.p, t2, sizeof(double) * n_t2, cudaMemcpyHostToDevice, st));
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_ovvv.p, ints->ovvv, sizeof(double) * n_ovvv, cudaMemcpyHostToDevice, st));
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_ovoo.p, ints->ovoo, sizeof(double) * n_ovoo, cudaMemcpyHostToDevice, st));
    TC_CUDA(ctx, cudaMemcpyAsync(ctx->in_ovov.p, ints->ovov, sizeof(double) * n_ovov, cudaMemcpyHostToDevice, st));
    s = run_device(ctx, o, v, in, prec, slices, e_ijk_dev, st, out);
  }
  if (s != TC_OK) return s;
  if (e_ijk) {
    TC_CUDA(ctx, cudaMemcpyAsync(e_ijk, e_ijk_dev, sizeof(double) * (size_t)o * o * o, cudaMemcpyDeviceToHost, st));
    TC_CUDA(ctx, cudaStreamSynchronize(st));
  }
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out->tflops_alg = alg_flops(o, v) / std::max(out->seconds, 1e-12) / 1e12;
  return TC_OK;
}

}  // extern "C"
