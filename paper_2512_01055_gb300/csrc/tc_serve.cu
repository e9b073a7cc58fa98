// Serving engine: continuous batching of many (T) jobs on one device
// (tc_submit / tc_poll / tc_wait / tc_cancel of include/tc.h).
//
// Two host threads per context:
//   * the admission worker takes queued jobs in arrival order while fewer than
//     max_inflight are admitted and their summed device footprint fits the
//     budget, allocates each job's device block from the stream-ordered pool,
//     copies host inputs, uploads its work tables and (split path) builds its
//     BF16 operand images, all on the job's own stream, then records an event;
//   * the scheduler runs iterations: it picks a precision group (FP64 or split
//     with s slices) round robin, gives every ready job of that group a slice
//     of its remaining work items (a fair share of an item budget sized to
//     about iteration_ms), and replays the group's CUDA graph -- one
//     persistent multi-job kernel over all those slices -- after updating the
//     kernel node's parameters.  Jobs whose last items ran are reduced in one
//     multi-job reduction and completed.
// Because every job keeps its own partial sums, a job's energy is the same
// bits whatever it was batched with.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tc_ctx.h"
#include "tc_internal.cuh"
#include "tc_plan.cuh"

namespace tc {
namespace {

using Clock = std::chrono::steady_clock;
constexpr int N_GROUPS = 4;               // 0: FP64, 1..3: split with 2..4 slices

enum class St { Queued, Prep, Ready, Done, Failed, Cancelled };

struct Req {
  uint64_t id = 0;
  int o = 0, v = 0, prec = 0, slices = 0, group = 0;
  bool dev_inputs = false;
  int nq = 0;                             // > 0: integrals from the DF factors (Eq. 6)
  std::vector<double> host[6];            // copies of host inputs (eps, t1, t2, ovvv, ovoo, ovov; B in [3] for DF)
  const double *din[6] = {};              // device inputs used by the kernels
  const double *dB = nullptr;             // DF factors on the device
  char *mem = nullptr;                    // device block: [host inputs][DF integrals][DF scratch][workspace][split images]
  size_t footprint = 0;
  size_t off_ints = 0, off_df = 0;        // DF jobs: assembled integrals and assembly scratch in the block
  Dims d{};
  plan::Layout L{};
  SplitLayout SL{};
  size_t off_ws = 0, off_split = 0;
  Work w{};
  cudaStream_t st = nullptr;
  cudaEvent_t ready = nullptr;
  bool waited = false;                    // the compute stream waits on `ready` once
  long long units = 0;                    // work units: FP64 items, or split-path triplets
  long long next_item = 0;                // next unit to run
  double cost_per_item = 1.0;             // cost of one unit
  St state = St::Queued;
  tc_status status = TC_OK;
  tc_result res{};
  Clock::time_point t_submit, t_start, t_done;
  bool started = false;
  bool inject_alloc_fault = false;        // test hook: treat this job's allocation as failed
};

double alg_flops(int o, int v) {
  const double O = o, V = v;
  return 2.0 * (O * O * O * V * V * V * V + O * O * O * O * V * V * V);
}

}  // namespace

struct Server {
  tc_ctx *ctx = nullptr;
  std::mutex mu;
  std::condition_variable cv_admit, cv_sched, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> active;               // admitted, not finished
  std::unordered_map<uint64_t, std::shared_ptr<Req>> table;
  uint64_t next_id = 1;
  size_t reserved = 0;
  bool stop = false;
  std::thread admit_th, sched_th;
  cudaStream_t compute = nullptr;
  std::vector<cudaStream_t> prep_streams;
  unsigned *d_counter = nullptr;          // FP64 work counter (zeroed by the graph)
  int *d_err = nullptr;                   // split kernels' wait-limit flag
  double *h_out = nullptr;                // pinned: 4 doubles per job of a reduction + err
  double *d_out = nullptr;                // device: 4 doubles per job of a reduction (E, sum |e|, E[5]_ST)
  cudaGraph_t graph[N_GROUPS] = {};
  cudaGraphExec_t exec[N_GROUPS] = {};
  cudaGraphNode_t knode[N_GROUPS][SPLIT_WT_LAUNCHES] = {};   // FP64 group: [0] only; split: the W-term chain
  cudaGraphNode_t enode[N_GROUPS] = {};   // split groups: the energy launch after the W-term launches
  double rate[N_GROUPS] = {3e7, 4e8, 3e8, 2e8};   // cost units per second (refined as iterations run)
  int rr = 0;                             // round-robin cursor over groups
  int fault_alloc = 0, fault_stall_ms = 0;
  tc_serve_stats stats{};
  int fp64_per_sm = 1;

  tc_status setup();
  void admit_loop();
  void sched_loop();
  void start_prep(const std::shared_ptr<Req> &r);
  bool run_iteration(int g, std::vector<std::shared_ptr<Req>> &jobs);
  void finish(std::vector<std::shared_ptr<Req>> &done);
  void fail_job(const std::shared_ptr<Req> &r, tc_status s);
};

namespace {

int group_of(int prec, int slices) { return prec == TC_FP64 ? 0 : slices - 1; }

}  // namespace

tc_status Server::setup() {
  cudaSetDevice(ctx->device);
  if (cudaStreamCreateWithFlags(&compute, cudaStreamNonBlocking) != cudaSuccess) return TC_ECUDA;
  prep_streams.resize(ctx->max_inflight);
  for (auto &s : prep_streams)
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return TC_ECUDA;
  if (cudaMalloc(&d_counter, 256) != cudaSuccess || cudaMalloc(&d_err, 256) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(double) * 4 * MAX_BATCH) != cudaSuccess ||
      cudaMallocHost(&h_out, sizeof(double) * (4 * MAX_BATCH + 1)) != cudaSuccess)
    return TC_ECUDA;
  cudaMemset(d_err, 0, 256);
  // keep freed job memory in the pool for reuse instead of returning it to the driver
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (fp64_blocks_per_sm(&fp64_per_sm) != cudaSuccess) return TC_ECUDA;
  admit_th = std::thread([this] { admit_loop(); });
  sched_th = std::thread([this] { sched_loop(); });
  return TC_OK;
}

void Server::fail_job(const std::shared_ptr<Req> &r, tc_status s) {
  // caller holds mu
  r->status = s;
  r->state = St::Failed;
  r->t_done = Clock::now();
  ++stats.failed;
}

// Allocation, copies, tables and BF16 images of one admitted job, on its stream.
void Server::start_prep(const std::shared_ptr<Req> &r) {
  Req &q = *r;
  const bool split = q.prec == TC_SPLIT_BF16;
  cudaError_t e = cudaSuccess;
  if (q.inject_alloc_fault) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&q.mem, q.footprint, q.st);
  if (e != cudaSuccess) {
    q.mem = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    reserved -= q.footprint;
    fail_job(r, TC_ENOMEM);
    active.erase(std::find(active.begin(), active.end(), r));
    cv_done.notify_all();
    cv_admit.notify_all();
    return;
  }
  if (!q.dev_inputs) {
    const size_t O = q.o, V = q.v;
    const size_t n[6] = {O + V, O * V, O * O * V * V, O * V * V * V, O * V * O * O, O * V * O * V};
    const int narr = q.nq > 0 ? 4 : 6;    // DF: eps, t1, t2, B
    size_t off = 0;
    for (int a = 0; a < narr; ++a) {
      double *dst = (double *)(q.mem + off);
      const size_t cnt = (q.nq > 0 && a == 3) ? q.host[3].size() : n[a];
      cudaMemcpyAsync(dst, q.host[a].data(), cnt * sizeof(double), cudaMemcpyHostToDevice, q.st);
      if (q.nq > 0 && a == 3) q.dB = dst;
      else q.din[a] = dst;
      off += cnt * sizeof(double);
    }
  }
  if (q.nq > 0) {
    // the integral blocks from the factors, in the job's block (Eq. 6)
    const size_t O = q.o, V = q.v;
    double *ovvv = (double *)(q.mem + q.off_ints), *ovoo = ovvv + O * V * V * V, *ovov = ovoo + O * V * O * O;
    int digits = 0;
    e = df_assemble(q.dB, q.nq, q.o, q.v, ovvv, ovoo, ovov, q.mem + q.off_df, ctx->num_sms, q.st, &digits);
    q.din[3] = ovvv;
    q.din[4] = ovoo;
    q.din[5] = ovov;
    q.res.df_digits = digits;
    if (e == cudaSuccess) {
      int derr = 0;
      e = cudaMemcpyAsync(&derr, df_error_flag(q.mem + q.off_df, q.o, q.v, q.nq), sizeof(int), cudaMemcpyDeviceToHost,
                          q.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(q.st);
      if (e == cudaSuccess && derr != 0) e = cudaErrorLaunchTimeout;
    }
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(mu);
      for (auto &h : q.host) std::vector<double>().swap(h);
      fail_job(r, e == cudaErrorLaunchTimeout ? TC_ETIMEOUT : TC_ECUDA);
      return;                             // memory released by the scheduler's sweep
    }
  }
  char *base = q.mem + q.off_ws;
  const std::vector<int4> tab = plan::tables(q.d, q.L, nullptr);
  cudaMemcpyAsync(base + q.L.trip, tab.data(), tab.size() * sizeof(int4), cudaMemcpyHostToDevice, q.st);
  q.w.trip = (const int4 *)(base + q.L.trip);
  q.w.orb = (const int4 *)(base + q.L.orb);
  q.w.partial = (double *)(base + q.L.partial);
  q.w.counter = (unsigned *)(base + q.L.counter);
  q.w.err = (int *)(base + q.L.counter + sizeof(unsigned));
  cudaMemsetAsync(q.w.counter, 0, 2 * sizeof(unsigned), q.st);
  if (split) {
    const Inputs in{q.din[0], q.din[1], q.din[2], q.din[3], q.din[4], q.din[5]};
    launch_split_prep(q.SL, in, q.mem + q.off_split, q.st);
  }
  cudaEventRecord(q.ready, q.st);
  e = cudaStreamSynchronize(q.st);        // the copies read the job's host vectors
  std::lock_guard<std::mutex> lk(mu);
  for (auto &h : q.host) std::vector<double>().swap(h);
  if (e != cudaSuccess) {
    fail_job(r, TC_ECUDA);
    return;                               // memory released by the scheduler's sweep
  }
  q.state = St::Ready;
  cv_sched.notify_all();
}

void Server::admit_loop() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    std::shared_ptr<Req> r;
    if (!queue.empty() && (int)active.size() < ctx->max_inflight &&
        reserved + queue.front()->footprint <= ctx->budget) {
      r = queue.front();
      queue.pop_front();
      r->inject_alloc_fault = fault_alloc != 0;
      fault_alloc = 0;
      reserved += r->footprint;
      r->state = St::Prep;
      int slot = 0;                       // a prep stream not used by another admitted job
      for (; slot < (int)prep_streams.size(); ++slot) {
        bool used = false;
        for (auto &a : active) used |= (a->st == prep_streams[slot]);
        if (!used) break;
      }
      r->st = prep_streams[slot % prep_streams.size()];
      active.push_back(r);
    }
    if (!r) {
      cv_admit.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    lk.unlock();
    start_prep(r);
    lk.lock();
  }
}

// One batched launch of group g over slices of `jobs` (all ready).
bool Server::run_iteration(int g, std::vector<std::shared_ptr<Req>> &jobs) {
  const int nj = (int)jobs.size();
  // water-filling: every job gets up to an equal share of the cost budget
  double budget = rate[g] * 1e-3 * ctx->iteration_ms;
  std::vector<long long> take(nj, 0);
  std::vector<int> open(nj);
  for (int j = 0; j < nj; ++j) open[j] = j;
  while (!open.empty() && budget > 0) {
    const double share = budget / open.size();
    std::vector<int> still;
    for (int j : open) {
      Req &q = *jobs[j];
      // split jobs run at most one block of triplets (the W buffer) per launch
      const long long cap = g == 0 ? q.units : q.SL.g.nb;
      const long long rem = std::min(q.units - q.next_item, cap) - take[j];
      const long long want = std::max<long long>(1, (long long)(share / q.cost_per_item));
      const long long t = std::min(rem, want);
      take[j] += t;
      budget -= t * q.cost_per_item;
      if (rem - t > 0 && t == want) still.push_back(j);
    }
    if (still.size() == open.size() && budget <= 0) break;
    open.swap(still);
  }
  for (int j = 0; j < nj; ++j) {
    Req &q = *jobs[j];
    if (!q.waited) { cudaStreamWaitEvent(compute, q.ready, 0); q.waited = true; }
    if (!q.started) { q.started = true; q.t_start = Clock::now(); }
  }
  void *args[SPLIT_WT_LAUNCHES], *eargs[1];
  cudaKernelNodeParams kp[SPLIT_WT_LAUNCHES] = {}, ep{};
  static thread_local FpBatch fb;
  static thread_local WtBatch wb[SPLIT_WT_LAUNCHES];
  static thread_local EnBatch eb;
  long long total = 0;
  double cost = 0;
  cudaError_t e = cudaSuccess;
  if (g == 0) {
    fb = FpBatch{};
    fb.njobs = nj;
    fb.counter = d_counter;
    for (int j = 0; j < nj; ++j) {
      Req &q = *jobs[j];
      const Inputs in{q.din[0], q.din[1], q.din[2], q.din[3], q.din[4], q.din[5]};
      fb.job[j] = FpJob{q.d, in, q.w, total, q.next_item};
      total += take[j];
      cost += take[j] * q.cost_per_item;
    }
    fb.total_items = total;
    const long long grid = std::min<long long>((long long)ctx->num_sms * fp64_per_sm, total);
    fp64_node_params(fb, (int)grid, args, &kp[0]);
  } else {
    wb[0] = WtBatch{};
    eb = EnBatch{};
    wb[0].njobs = eb.njobs = nj;
    wb[0].err = eb.err = d_err;
    for (int j = 0; j < nj; ++j) {
      Req &q = *jobs[j];
      const Inputs in{q.din[0], q.din[1], q.din[2], q.din[3], q.din[4], q.din[5]};
      const int t0 = (int)q.next_item, nt = (int)take[j];
      wb[0].job[j] = wt_job(q.SL, q.mem + q.off_split, q.w.trip, t0, nt);
      if (e == cudaSuccess) e = en_job(&eb.job[j], q.d, q.SL, q.mem + q.off_split, in, q.w, t0, nt);
      total += take[j];
      cost += take[j] * q.cost_per_item;
    }
    if (e == cudaSuccess) e = split_block_params(wb, eb, g + 1, ctx->num_sms, args, eargs, kp, &ep);
  }
  if (e != cudaSuccess) return false;
  if (!exec[g]) {
    // the group's graph: FP64, [zero the work counter] -> [multi-job kernel];
    // split, [W-term F0] -> [F1] -> [F2] -> [energy]
    e = cudaGraphCreate(&graph[g], 0);
    cudaGraphNode_t mnode = nullptr;
    if (e == cudaSuccess && g == 0) {
      cudaMemsetParams mp{};
      mp.dst = d_counter;
      mp.value = 0;
      mp.elementSize = 4;
      mp.width = 1;
      mp.height = 1;
      e = cudaGraphAddMemsetNode(&mnode, graph[g], nullptr, 0, &mp);
    }
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&knode[g][0], graph[g], mnode ? &mnode : nullptr, mnode ? 1 : 0, &kp[0]);
    if (g != 0) {
      for (int f = 1; f < SPLIT_WT_LAUNCHES && e == cudaSuccess; ++f)
        e = cudaGraphAddKernelNode(&knode[g][f], graph[g], &knode[g][f - 1], 1, &kp[f]);
      if (e == cudaSuccess) e = cudaGraphAddKernelNode(&enode[g], graph[g], &knode[g][SPLIT_WT_LAUNCHES - 1], 1, &ep);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec[g], graph[g], 0);
  } else {
    e = cudaGraphExecKernelNodeSetParams(exec[g], knode[g][0], &kp[0]);
    if (g != 0) {
      for (int f = 1; f < SPLIT_WT_LAUNCHES && e == cudaSuccess; ++f)
        e = cudaGraphExecKernelNodeSetParams(exec[g], knode[g][f], &kp[f]);
      if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(exec[g], enode[g], &ep);
    }
  }
  const auto t0 = Clock::now();
  if (e == cudaSuccess) e = cudaGraphLaunch(exec[g], compute);
  if (e == cudaSuccess) e = cudaStreamSynchronize(compute);
  const double sec = std::chrono::duration<double>(Clock::now() - t0).count();
  int errflag = 0;
  if (e == cudaSuccess && g != 0) {
    e = cudaMemcpy(&errflag, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (errflag) cudaMemset(d_err, 0, sizeof(int));
  }
  std::lock_guard<std::mutex> lk(mu);
  ++stats.iterations;
  ++stats.graph_launches;
  stats.batched_jobs += nj;
  if (e != cudaSuccess || errflag) {
    for (auto &r : jobs) fail_job(r, errflag ? TC_ETIMEOUT : TC_ECUDA);
    return false;
  }
  if (sec > 1e-4) rate[g] = 0.5 * rate[g] + 0.5 * cost / sec;
  for (int j = 0; j < nj; ++j) jobs[j]->next_item += take[j];
  return true;
}

// Multi-job reduction of the jobs whose last items ran, then completion.
void Server::finish(std::vector<std::shared_ptr<Req>> &done) {
  for (size_t b0 = 0; b0 < done.size(); b0 += MAX_BATCH) {
    const int n = (int)std::min<size_t>(MAX_BATCH, done.size() - b0);
    RedBatch rb{};
    rb.njobs = n;
    for (int j = 0; j < n; ++j) {
      Req &q = *done[b0 + j];
      char *base = q.mem + q.off_ws;
      rb.job[j] = RedJob{q.d.n_trip, q.d.items_per_trip, q.o, q.w.trip, q.w.partial,
                         (double *)(base + q.L.e_trip), nullptr, d_out + 4 * j};
    }
    cudaError_t e = launch_reduce(rb, compute);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_out, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, compute);
    for (int j = 0; j < n; ++j) cudaFreeAsync(done[b0 + j]->mem, compute);
    if (e == cudaSuccess) e = cudaStreamSynchronize(compute);
    std::lock_guard<std::mutex> lk(mu);
    for (int j = 0; j < n; ++j) {
      auto &r = done[b0 + j];
      r->mem = nullptr;
      reserved -= r->footprint;
      active.erase(std::find(active.begin(), active.end(), r));
      if (e != cudaSuccess) { fail_job(r, TC_ECUDA); continue; }
      r->t_done = Clock::now();
      r->res.e_t = h_out[4 * j];
      r->res.e_t5 = h_out[4 * j + 2];
      r->state = St::Done;
      r->status = TC_OK;
      ++stats.completed;
    }
    cv_done.notify_all();
    cv_admit.notify_all();
  }
}

void Server::sched_loop() {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    if (fault_stall_ms > 0) {
      const int ms = fault_stall_ms;
      fault_stall_ms = 0;
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::milliseconds(ms));
      lk.lock();
    }
    // release jobs that failed during preparation
    for (size_t a = 0; a < active.size();) {
      auto r = active[a];
      if (r->state == St::Failed) {
        if (r->mem) { cudaFreeAsync(r->mem, r->st); r->mem = nullptr; }
        reserved -= r->footprint;
        active.erase(active.begin() + a);
        cv_done.notify_all();
        cv_admit.notify_all();
      } else {
        ++a;
      }
    }
    // pick the next group (round robin) that has ready work
    std::vector<std::shared_ptr<Req>> jobs;
    int g = -1;
    for (int k = 0; k < N_GROUPS && g < 0; ++k) {
      const int gg = (rr + k) % N_GROUPS;
      for (auto &r : active)
        if (r->group == gg && r->state == St::Ready && r->next_item < r->units && (int)jobs.size() < MAX_BATCH)
          jobs.push_back(r);
      if (!jobs.empty()) g = gg;
    }
    // jobs with no items at all (o = 1 or v too small to matter) complete directly
    std::vector<std::shared_ptr<Req>> done;
    for (auto &r : active)
      if (r->state == St::Ready && r->next_item >= r->units) { done.push_back(r); r->state = St::Prep; }
    if (g < 0 && done.empty()) {
      cv_sched.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    rr = (g < 0 ? rr : g) + 1;
    lk.unlock();
    if (g >= 0) {
      run_iteration(g, jobs);
      for (auto &r : jobs)
        if (r->state == St::Ready && r->next_item >= r->units) { done.push_back(r); r->state = St::Prep; }
    }
    if (!done.empty()) {
      for (auto &r : done)
        if (!r->waited) { cudaStreamWaitEvent(compute, r->ready, 0); r->waited = true; }
      finish(done);
    }
    lk.lock();
  }
}

void server_destroy(Server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_admit.notify_all();
  s->cv_sched.notify_all();
  if (s->admit_th.joinable()) s->admit_th.join();
  if (s->sched_th.joinable()) s->sched_th.join();
  cudaSetDevice(s->ctx->device);
  cudaDeviceSynchronize();
  for (auto &r : s->active)
    if (r->mem) cudaFree(r->mem);
  for (auto &kv : s->table)
    if (kv.second->ready) cudaEventDestroy(kv.second->ready);
  for (int g = 0; g < N_GROUPS; ++g) {
    if (s->exec[g]) cudaGraphExecDestroy(s->exec[g]);
    if (s->graph[g]) cudaGraphDestroy(s->graph[g]);
  }
  for (auto st : s->prep_streams) if (st) cudaStreamDestroy(st);
  if (s->compute) cudaStreamDestroy(s->compute);
  if (s->d_counter) cudaFree(s->d_counter);
  if (s->d_err) cudaFree(s->d_err);
  if (s->d_out) cudaFree(s->d_out);
  if (s->h_out) cudaFreeHost(s->h_out);
  delete s;
}

}  // namespace tc

namespace {

tc_status get_server(tc_ctx *ctx, tc::Server **out) {
  std::lock_guard<std::mutex> lk(ctx->serve_mu);
  if (!ctx->server) {
    auto *s = new (std::nothrow) tc::Server();
    if (!s) return TC_ENOMEM;
    s->ctx = ctx;
    const tc_status st = s->setup();
    if (st != TC_OK) { tc::server_destroy(s); return st; }
    ctx->server = s;
  }
  *out = ctx->server;
  return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_submit(tc_ctx *ctx, const tc_job *job, uint64_t *ticket) {
  if (!ctx || !job || !ticket) return TC_EINVAL;
  const int o = job->o, v = job->v;
  int prec = job->prec < 0 ? ctx->default_prec : job->prec;
  int slices = job->slices <= 0 ? ctx->default_slices : job->slices;
  if (o <= 0 || v <= 0 || (long long)o * v * v * v > (1LL << 40)) return TC_EINVAL;
  if (job->nq < 0 || !job->eps || !job->t1 || !job->t2) return TC_EINVAL;
  if (job->nq > 0 ? !job->B : (!job->ints.ovvv || !job->ints.ovoo || !job->ints.ovov)) return TC_EINVAL;
  if (prec != TC_FP64 && prec != TC_SPLIT_BF16) return TC_EINVAL;
  if (prec == TC_SPLIT_BF16 && (slices < 2 || slices > 4)) return TC_EINVAL;
  if (prec == TC_FP64) slices = 0;
  tc::Server *s = nullptr;
  tc_status st = get_server(ctx, &s);
  if (st != TC_OK) return st;
  auto r = std::make_shared<tc::Req>();
  r->o = o;
  r->v = v;
  r->prec = prec;
  r->slices = slices;
  r->group = tc::group_of(prec, slices);
  r->dev_inputs = (job->flags & TC_JOB_DEVICE_INPUTS) != 0;
  const bool split = prec == TC_SPLIT_BF16;
  r->d = split ? tc::plan::make_dims(o, v, tc::split_tile(), -1, tc::split_orb_per_item(o, v, slices))
              : tc::plan::make_dims(o, v, tc::fp64_tile());
  r->L = tc::plan::make_layout(r->d);
  if (split) r->SL = tc::split_layout(o, v, slices);
  r->nq = job->nq;
  const size_t O = o, V = v, NB = (size_t)job->nq * (O + V) * (O + V);
  const size_t ints_b = sizeof(double) * (O * V * V * V + O * V * O * O + O * V * O * V);
  // [host inputs][DF integrals][DF scratch][workspace][split images]
  const size_t in_b = r->dev_inputs ? 0
                      : tc::plan::align256(r->nq > 0 ? sizeof(double) * (O + V + O * V + O * O * V * V + NB)
                                                     : tc::plan::input_bytes(o, v));
  r->off_ints = in_b;
  r->off_df = r->off_ints + (r->nq > 0 ? tc::plan::align256(ints_b) : 0);
  r->off_ws = r->off_df + (r->nq > 0 ? tc::plan::align256(tc::df_scratch_bytes(o, v, r->nq)) : 0);
  r->off_split = r->off_ws + r->L.total;
  r->footprint = r->off_split + r->SL.total;
  // cost units: one orbit's worth of K values; a split unit is a whole triplet
  r->units = split ? r->d.n_trip : r->d.n_items;
  r->cost_per_item = (double)(split ? r->d.n_orb : r->d.orb_per_item) * (v + 16.0 * ((o + 15) / 16));
  if (r->footprint > ctx->budget) return TC_ENOMEM;
  const double *src[6] = {job->eps, job->t1, job->t2, job->ints.ovvv, job->ints.ovoo, job->ints.ovov};
  const size_t n[6] = {O + V, O * V, O * O * V * V, O * V * V * V, O * V * O * O, O * V * O * V};
  const int narr = r->nq > 0 ? 3 : 6;
  if (r->dev_inputs) {
    for (int a = 0; a < narr; ++a) r->din[a] = src[a];
    if (r->nq > 0) r->dB = job->B;
  } else {
    for (int a = 0; a < narr; ++a) r->host[a].assign(src[a], src[a] + n[a]);
    if (r->nq > 0) r->host[3].assign(job->B, job->B + NB);
  }
  if (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess) return TC_ECUDA;
  r->res.o = o;
  r->res.v = v;
  r->res.prec = prec;
  r->res.slices = slices;
  r->t_submit = tc::Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if ((int)s->queue.size() >= ctx->max_queue) {
      cudaEventDestroy(r->ready);
      return TC_EBUSY;
    }
    r->id = s->next_id++;
    s->table[r->id] = r;
    s->queue.push_back(r);
    ++s->stats.submitted;
    *ticket = r->id;
  }
  s->cv_admit.notify_all();
  return TC_OK;
}

static tc_status collect(tc::Server *s, std::unordered_map<uint64_t, std::shared_ptr<tc::Req>>::iterator it,
                         tc_result *out) {
  // caller holds s->mu; the job is finished
  auto r = it->second;
  if (out) {
    *out = r->res;
    out->seconds = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    out->queue_seconds = r->started ? std::chrono::duration<double>(r->t_start - r->t_submit).count() : out->seconds;
    out->n_items = r->d.n_items;
    out->tflops_alg = tc::alg_flops(r->o, r->v) / std::max(out->seconds, 1e-12) / 1e12;
  }
  const tc_status st = r->state == tc::St::Cancelled ? TC_ECANCELLED : r->status;
  if (r->ready) cudaEventDestroy(r->ready);
  r->ready = nullptr;
  s->table.erase(it);
  return st;
}

tc_status tc_poll(tc_ctx *ctx, uint64_t ticket, tc_result *out) {
  if (!ctx || !ctx->server) return TC_EINVAL;
  tc::Server *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return TC_EINVAL;
  const tc::St st = it->second->state;
  if (st != tc::St::Done && st != tc::St::Failed && st != tc::St::Cancelled) return TC_ENOTREADY;
  return collect(s, it, out);
}

tc_status tc_wait(tc_ctx *ctx, uint64_t ticket, int timeout_ms, tc_result *out) {
  if (!ctx || !ctx->server) return TC_EINVAL;
  tc::Server *s = ctx->server;
  if (timeout_ms < 0) timeout_ms = ctx->timeout_ms;
  const auto deadline = tc::Clock::now() + std::chrono::milliseconds(timeout_ms);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return TC_EINVAL;
    const tc::St st = it->second->state;
    if (st == tc::St::Done || st == tc::St::Failed || st == tc::St::Cancelled) return collect(s, it, out);
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto it2 = s->table.find(ticket);
      if (it2 == s->table.end()) return TC_EINVAL;
      const tc::St st2 = it2->second->state;
      if (st2 == tc::St::Done || st2 == tc::St::Failed || st2 == tc::St::Cancelled) return collect(s, it2, out);
      return TC_ETIMEOUT;
    }
  }
}

tc_status tc_cancel(tc_ctx *ctx, uint64_t ticket) {
  if (!ctx || !ctx->server) return TC_EINVAL;
  tc::Server *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return TC_EINVAL;
  auto r = it->second;
  if (r->state != tc::St::Queued) return TC_EBUSY;
  s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  r->state = tc::St::Cancelled;
  r->t_done = tc::Clock::now();
  ++s->stats.cancelled;
  s->cv_done.notify_all();
  return TC_OK;
}

tc_status tc_serve_stats_get(tc_ctx *ctx, tc_serve_stats *out) {
  if (!ctx || !out) return TC_EINVAL;
  std::memset(out, 0, sizeof *out);
  if (!ctx->server) return TC_OK;
  tc::Server *s = ctx->server;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = s->queue.size();
  out->inflight = s->active.size();
  out->reserved_bytes = s->reserved;
  return TC_OK;
}

tc_status tc_inject_fault(tc_ctx *ctx, int kind, int param) {
  if (!ctx) return TC_EINVAL;
  tc::Server *s = nullptr;
  tc_status st = get_server(ctx, &s);
  if (st != TC_OK) return st;
  std::lock_guard<std::mutex> lk(s->mu);
  if (kind == TC_FAULT_ALLOC) s->fault_alloc = 1;
  else if (kind == TC_FAULT_STALL) s->fault_stall_ms = param > 0 ? param : 0;
  else return TC_EINVAL;
  return TC_OK;
}

}  // extern "C"
