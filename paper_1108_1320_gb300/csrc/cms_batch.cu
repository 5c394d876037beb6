// cms_batch.cu - many compressed products in one persistent launch.
//
// A batch is a fixed list of instances (A, B, shapes, storage type, hashes,
// output).  Creating it plans every instance (optionally autotuning the
// inner-index chunking and the generic kernel's group size against the
// instance's own data), lays out all workspaces in one allocation,
// computes the constant twiddle tables and uploads one task descriptor per
// instance.  Running it launches:
//   * the front-end twiddles of instances served by the generic kernel,
//   * ONE persistent kernel over the tasks of every instance (longest
//     first), and
//   * per instance, the fixed-order reduction and inverse FFT.
// cms_batch_run_graph captures that sequence once in a CUDA graph and
// replays it.
#include <atomic>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include <unistd.h>

#include "cms_internal.h"

struct cms_batch {
  int device = 0;
  std::vector<cms_instance> items;
  std::vector<cms::SketchPlan> plans;
  std::vector<size_t> ws_off;       // workspace offset of each instance
  std::vector<int> order;           // instance order in the persistent launch
  char* ws = nullptr;
  size_t ws_bytes = 0;
  void* d_desc = nullptr;
  int* d_start = nullptr;
  int* d_next = nullptr;
  int total_tasks = 0;
  size_t smem = 0;
  int grid = 0;
  int launches = 0;
  int use_tmem = 0;   // some instance keeps its twiddle records in tensor memory
  void* d_inv = nullptr;            // arguments of the batched reduction + inverse
  cms::InverseBatch inv;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
};

namespace cms {
namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

std::string tune_key(const cms_instance& it, const SketchPlan& p, int sms) {
  std::ostringstream k;
  k << "b=" << p.b << ",n1=" << it.n1 << ",n2=" << it.n2 << ",n3=" << it.n3 << ",dt=" << it.dt
    << ",d=" << p.d << ",sms=" << sms << ",kernel=" << (p.fast ? "fast" : "generic")
    << (p.alias ? "-alias" : "");
  return k.str();
}

struct Tuned {
  int nkc = 0, G = 0;
  double ms = 0.0;
};

// The cache file holds one line per key:  key nkc G ms
std::map<std::string, Tuned> load_cache(const char* path) {
  std::map<std::string, Tuned> m;
  if (!path) return m;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string key;
    Tuned t;
    if (is >> key >> t.nkc >> t.G >> t.ms) m[key] = t;
  }
  return m;
}

// Written to a temporary file beside it and renamed over it, so that a
// reader (or another process) never sees a partly written cache; the cache
// only saves tuning time, so a failed write is dropped.
void save_cache(const char* path, const std::map<std::string, Tuned>& m) {
  if (!path) return;
  // process id and a process-wide counter: two batches tuning on different
  // host threads of one process never write the same temporary file
  static std::atomic<unsigned long long> serial{0};
  const std::string tmp = std::string(path) + ".tmp." + std::to_string(static_cast<long long>(getpid())) + "." +
                          std::to_string(serial.fetch_add(1));
  {
    std::ofstream f(tmp, std::ios::trunc);
    if (!f) return;
    for (const auto& kv : m)
      f << kv.first << " " << kv.second.nkc << " " << kv.second.G << " " << kv.second.ms << "\n";
    f.flush();
    if (!f) {
      std::remove(tmp.c_str());
      return;
    }
  }
  if (std::rename(tmp.c_str(), path) != 0) std::remove(tmp.c_str());
}

int num_sms(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

size_t smem_optin(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? static_cast<size_t>(v) : 48 * 1024;
}

cms_status fail(cms_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

cms_status cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return CMS_ERR_CUDA;
}

// Time one configuration of one instance with the single-instance launch.
cudaError_t time_plan(const SketchPlan& p, const cms_instance& it, char* ws, cudaStream_t s, double* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess)
    e = launch_sketch(p, it.h, it.A, it.lda, it.B, it.ldb, it.n1, it.n2, it.n3, it.dt, it.c, ws, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  for (int r = 0; r < 2 && e == cudaSuccess; ++r)
    e = launch_sketch(p, it.h, it.A, it.lda, it.B, it.ldb, it.n1, it.n2, it.n3, it.dt, it.c, ws, s);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  *ms = t / 2.0;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

void release(cms_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->ws) cudaFree(b->ws);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_start) cudaFree(b->d_start);
  if (b->d_next) cudaFree(b->d_next);
  if (b->d_inv) cudaFree(b->d_inv);
  b->d_inv = nullptr;
  b->exec = nullptr;
  b->graph = nullptr;
  b->ws = nullptr;
  b->d_desc = nullptr;
  b->d_start = nullptr;
  b->d_next = nullptr;
}

}  // namespace
}  // namespace cms

using namespace cms;

extern "C" {

constexpr int kBatchWaves = 12;

// Work of an instance in conventional flops: d n2 5 b log2 b.
double instance_work(const cms_instance& it) {
  const double b = static_cast<double>(it.h->b);
  return static_cast<double>(it.h->d) * static_cast<double>(std::max<int64_t>(it.n2, 1)) * 5.0 * b *
         std::log2(std::max(b, 2.0));
}

// Chunks of instance `it` (planned as p) under the batch budget: tasks in
// proportion to its share of the batch's work, at least one per unit.
int batch_chunks(const cms_instance& it, const SketchPlan& p, const cms_instance* items, int count, int sms) {
  double total = 0.0;
  for (int i = 0; i < count; ++i) total += instance_work(items[i]);
  if (!(total > 0.0)) return 0;
  const double units = static_cast<double>(p.d) * (p.fast ? (p.nrows + 1) / 2 : p.nrows);
  const double tasks = static_cast<double>(kBatchWaves) * sms * instance_work(it) / total;
  return std::max(1, static_cast<int>(std::lround(tasks / std::max(units, 1.0))));
}

cms_status cms_batch_create(const cms_instance* items, int32_t count, int32_t flags,
                            const char* tune_cache, void* stream, cms_batch** out) {
  NvtxRange nvtx_range("cms_batch_create");
  if (!out) return fail(CMS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !items) return fail(CMS_ERR_INVALID_ARG, "need at least one instance");
  cms_batch* b = new cms_batch();
  cudaGetDevice(&b->device);
  const int sms = num_sms(b->device);
  const size_t optin = smem_optin(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  b->items.assign(items, items + count);
  b->plans.resize(count);
  b->ws_off.resize(count);
  std::string why;
  // ---- plan every instance (tuned shapes come from the cache) ------------
  std::map<std::string, Tuned> cache = load_cache(tune_cache);
  bool cache_dirty = false;
  for (int i = 0; i < count; ++i) {
    const cms_instance& it = items[i];
    if (!it.h || !it.c) { delete b; return fail(CMS_ERR_INVALID_ARG, "instance with NULL hashes or c"); }
    if (it.h->device != b->device) { delete b; return fail(CMS_ERR_INVALID_ARG, "instances on another device"); }
    if (it.n1 < 0 || it.n2 < 0 || it.n3 < 0 || it.n1 > it.h->n || it.n3 > it.h->n ||
        it.lda < std::max<int64_t>(it.n1, 1) || it.ldb < std::max<int64_t>(it.n3, 1) ||
        (it.dt != CMS_F32 && it.dt != CMS_BF16 && it.dt != CMS_F64)) {
      delete b;
      return fail(CMS_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": bad shape, stride or dtype");
    }
    SketchPlan p;
    // the persistent batched kernel runs the lock-step fast body
    int r = make_sketch_plan(it.h, it.n1, it.n2, it.n3, it.dt, sms, optin, &p, &why, it.A, it.lda, it.B, it.ldb,
                             true, 0, 0, false, false);
    if (r != CMS_OK) { delete b; return fail(static_cast<cms_status>(r), "instance " + std::to_string(i) + ": " + why); }
    // k-chunking for the batch as a whole: each instance gets tasks in
    // proportion to its work out of a budget of kBatchWaves waves over the
    // SMs (the planner alone would split every instance to fill the GPU by
    // itself: many short tasks, each repeating its prologue and writing a
    // partial row)
    {
      const int nkc = batch_chunks(it, p, items, count, sms);
      SketchPlan q;
      if (nkc > 0 && make_sketch_plan(it.h, it.n1, it.n2, it.n3, it.dt, sms, optin, &q, &why, it.A, it.lda, it.B,
                                      it.ldb, true, nkc, 0, false, false) == CMS_OK)
        p = q;
    }
    auto hit = cache.find(tune_key(it, p, sms));
    if (hit != cache.end()) {
      SketchPlan q;
      if (make_sketch_plan(it.h, it.n1, it.n2, it.n3, it.dt, sms, optin, &q, &why, it.A, it.lda, it.B, it.ldb,
                           true, hit->second.nkc, hit->second.G, false, false) == CMS_OK)
        p = q;
    } else if (flags & CMS_BATCH_AUTOTUNE) {
      // candidates: the planner's chunking, half and twice as many chunks;
      // for the generic kernel also groups of 1, 2 and 4 inner indices
      std::vector<std::pair<int, int>> cand;
      for (int mul : {1, 2, 4}) {
        const int nk = std::max(1, p.nkc * mul / 2);
        if (p.fast) cand.push_back({nk, 0});
        else for (int g : {1, 2, 4}) cand.push_back({nk, g});
      }
      std::vector<SketchPlan> cps;
      size_t need = 0;
      for (auto& c2 : cand) {
        SketchPlan q;
        if (make_sketch_plan(it.h, it.n1, it.n2, it.n3, it.dt, sms, optin, &q, &why, it.A, it.lda, it.B,
                             it.ldb, true, c2.first, c2.second, false, false) == CMS_OK) {
          cps.push_back(q);
          need = std::max(need, q.ws_bytes);
        }
      }
      char* tws = nullptr;
      cudaError_t e = cudaMalloc(&tws, std::max<size_t>(need, 256));
      if (e != cudaSuccess) { delete b; return cuda_fail(e, "cms_batch_create (autotune workspace)"); }
      double best = 1e30;
      for (const SketchPlan& q : cps) {
        double ms = 0.0;
        e = time_plan(q, it, tws, s, &ms);
        if (e != cudaSuccess) { cudaFree(tws); delete b; return cuda_fail(e, "cms_batch_create (autotune)"); }
        if (ms < best) { best = ms; p = q; }
      }
      cudaFree(tws);
      cache[tune_key(it, p, sms)] = Tuned{p.nkc, p.fast ? 0 : p.G, best};
      cache_dirty = true;
    }
    b->plans[i] = p;
  }
  if (cache_dirty) save_cache(tune_cache, cache);
  // ---- one workspace for all instances ----------------------------------
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    b->ws_off[i] = off;
    off = align256(off + b->plans[i].ws_bytes);
  }
  b->ws_bytes = off;
  cudaError_t e = cudaMalloc(&b->ws, std::max<size_t>(off, 256));
  if (e != cudaSuccess) { release(b); delete b; return cuda_fail(e, "cms_batch_create (workspace)"); }
  // ---- task layout: instances with the longest tasks first --------------
  b->order.resize(count);
  for (int i = 0; i < count; ++i) b->order[i] = i;
  auto cost = [&](int i) {
    const SketchPlan& p = b->plans[i];
    const double per_k = static_cast<double>(p.C) * (p.fast ? 2.0 : 1.0);
    return per_k * static_cast<double>(p.kchunk) * (p.fast ? 0.2 : 1.0);
  };
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  const size_t dsz = batch_desc_bytes();
  std::vector<unsigned char> desc(dsz * count);
  std::vector<int> start(count);
  int total = 0;
  size_t smem = 0;
  for (int q = 0; q < count; ++q) {
    const int i = b->order[q];
    const cms_instance& it = items[i];
    const SketchPlan& p = b->plans[i];
    fill_batch_desc(desc.data() + dsz * q, p, it.h, it.A, it.lda, it.B, it.ldb, it.n1, it.n2, it.n3, it.dt,
                    b->ws + b->ws_off[i]);
    start[q] = total;
    total += batch_tasks(p);
    smem = std::max(smem, p.smem);
  }
  b->total_tasks = total;
  b->use_tmem = 0;
  for (const auto& p : b->plans) b->use_tmem |= (p.fast && p.tmem_rec) ? 1 : 0;
  if (b->use_tmem) smem = std::max(smem, kSmemOneBlockPerSm);
  b->smem = smem;
  b->grid = std::max(1, std::min(total, sms));
  if ((e = cudaMalloc(&b->d_desc, desc.size())) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void**>(&b->d_start), sizeof(int) * count)) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void**>(&b->d_next), sizeof(int))) != cudaSuccess ||
      (e = cudaMemcpy(b->d_desc, desc.data(), desc.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(b->d_start, start.data(), sizeof(int) * count, cudaMemcpyHostToDevice)) != cudaSuccess) {
    release(b);
    delete b;
    return cuda_fail(e, "cms_batch_create (descriptors)");
  }
  // constant twiddle tables of every instance
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const SketchPlan& p = b->plans[i];
    char* w = b->ws + b->ws_off[i];
    e = launch_twiddle_tables(reinterpret_cast<float2*>(w + p.off_twC), static_cast<int>(p.C),
                              reinterpret_cast<float2*>(w + p.off_twR), static_cast<int>(p.R), s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { release(b); delete b; return cuda_fail(e, "cms_batch_create (tables)"); }
  // every instance's reduction and inverse as two launches (rows, columns)
  {
    std::vector<InverseSpec> specs(count);
    for (int i = 0; i < count; ++i) {
      const SketchPlan& p = b->plans[i];
      char* w = b->ws + b->ws_off[i];
      specs[i] = InverseSpec{&p, reinterpret_cast<const float2*>(w + p.off_partial),
                             reinterpret_cast<float2*>(w + p.off_V), reinterpret_cast<const float2*>(w + p.off_twC),
                             reinterpret_cast<const float2*>(w + p.off_twR), items[i].c};
    }
    e = cudaMalloc(&b->d_inv, inverse_batch_bytes(count));
    if (e == cudaSuccess) e = build_inverse_batch(specs, b->d_inv, &b->inv, s);
    if (e != cudaSuccess) { release(b); delete b; return cuda_fail(e, "cms_batch_create (inverse arguments)"); }
  }
  int launches = 2 + 2;   // counter reset + persistent kernel + batched inverse (rows, columns)
  for (int i = 0; i < count; ++i) launches += b->plans[i].fast ? 0 : 1;
  b->launches = launches;
  *out = b;
  return CMS_OK;
}

cms_status cms_batch_run(cms_batch* b, void* stream) {
  NvtxRange nvtx_range("cms_batch_run");
  if (!b) return fail(CMS_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < b->items.size() && e == cudaSuccess; ++i)
    if (!b->plans[i].fast) e = launch_frontend_twiddles(b->plans[i], b->items[i].h, b->ws + b->ws_off[i], s);
  if (e == cudaSuccess)
    e = launch_sketch_batched(b->d_desc, b->d_start, static_cast<int>(b->items.size()), b->total_tasks,
                              b->d_next, b->smem, b->grid, b->use_tmem, s);
  if (e == cudaSuccess) e = launch_inverse_batched(b->inv, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_batch_run");
  return CMS_OK;
}

cms_status cms_batch_run_graph(cms_batch* b, void* stream) {
  NvtxRange nvtx_range("cms_batch_run_graph");
  if (!b) return fail(CMS_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return fail(CMS_ERR_INVALID_ARG, "graph capture needs a non-default stream");
  cudaError_t e = cudaSuccess;
  if (!b->exec) {
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cms_batch_run_graph (begin capture)");
    cms_status st = cms_batch_run(b, stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (st != CMS_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cms_batch_run_graph (end capture)");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(e, "cms_batch_run_graph (instantiate)"); }
    b->graph = g;
  }
  e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "cms_batch_run_graph (launch)");
  return CMS_OK;
}

cms_status cms_batch_info(const cms_batch* b, int32_t* instances, int32_t* tasks, int32_t* launches,
                          size_t* ws_bytes, int32_t* fast_instances) {
  if (!b) return fail(CMS_ERR_INVALID_ARG, "batch is NULL");
  if (instances) *instances = static_cast<int32_t>(b->items.size());
  if (tasks) *tasks = b->total_tasks;
  if (launches) *launches = b->launches;
  if (ws_bytes) *ws_bytes = b->ws_bytes;
  if (fast_instances) {
    int f = 0;
    for (const auto& p : b->plans) f += p.fast ? 1 : 0;
    *fast_instances = f;
  }
  return CMS_OK;
}

cms_status cms_batch_free(cms_batch* b) {
  if (!b) return CMS_OK;
  cudaDeviceSynchronize();
  release(b);
  delete b;
  return CMS_OK;
}

}  // extern "C"
