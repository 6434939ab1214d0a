// Sigma tile autotuner and the batched multi-geometry Davidson solve.
//
// Autotuner: for one (Hamiltonian, subspace, links) it times the sigma product for
// each candidate tile configuration -- rows per warp of the same-spin row products
// and, for the opposite-spin term, the alpha-single chunk width of the CUDA-core
// kernel or the form of the tensor-core kernel (pipeline depth 1 or 2, or the
// tile-stationary warp-specialised kernel) --
// and stores the fastest in the links handles.  Results are cached per problem
// class (orbitals, electrons, precision, and the string counts in quarter-octave
// buckets), so geometries of a scan with similar sizes are tuned once.
//
// Batched solve: the geometries of a scan are independent eigenproblems of uneven
// size.  In the lockstep form (the default) every geometry's Davidson runs on a host
// thread and a stream of its own, and hands each sigma product to a shared batcher:
// when every solve still running has handed in its product, the round runs as one
// batched launch per sigma stage over all of them -- for the tensor-core term a
// persistent kernel taking (geometry, alpha string) items from a device work queue --
// and each solve continues when its product is done.  A solve that has converged
// leaves the rounds.  The vector operations of the solves stay on their own streams
// and overlap.  In the worker form, the geometries are ordered by estimated cost
// (longest first) and handed out to n_streams worker threads, each driving the
// single-geometry Davidson on a stream of its own.
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "hinqs_internal.cuh"

namespace hinqs {

int check_triplet(const hinqs_ham_s* H, const hinqs_subspace_s* B, const hinqs_links_s* la,
                  const hinqs_links_s* lb, const char* who);

namespace {

using TuneKey = std::tuple<int, int, int, int, int, int>;
struct TuneVal {
  int rows, ch, stages;
  double ms;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneVal> g_tune_cache;

int bucket(int64_t n) { return (int)std::floor(4.0 * std::log2((double)std::max<int64_t>(n, 1))); }

__global__ void k_fill_pattern(void* x, int64_t N, int is_double) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / (1.0 + (double)(i % 97));
    if (is_double) static_cast<double*>(x)[i] = v;
    else static_cast<float*>(x)[i] = (float)v;
  }
}

}  // namespace

int autotune_impl(const hinqs_ham_s* H, const hinqs_subspace_s* B, hinqs_links_s* la,
                  hinqs_links_s* lb, int precision, double* best_ms, cudaStream_t s) {
  const TuneKey key{H->n, H->n_alpha, H->n_beta, precision, bucket(B->Na), bucket(B->Nb)};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      la->tune_rows = lb->tune_rows = it->second.rows;
      la->tune_ch = it->second.ch;
      la->tune_stages = it->second.stages;
      if (best_ms) *best_ms = it->second.ms;
      return HINQS_OK;
    }
  }
  const int64_t N = B->Na * B->Nb;
  const bool dbl = precision == HINQS_PREC_FP64;
  const size_t esz = dbl ? sizeof(double) : sizeof(float);
  void *c = nullptr, *sg = nullptr;
  if (cudaMallocAsync(&c, N * esz, s) != cudaSuccess || cudaMallocAsync(&sg, N * esz, s) != cudaSuccess) {
    cudaGetLastError();
    if (c) cudaFreeAsync(c, s);
    return fail(HINQS_ERR_OOM, "hinqs_autotune: no room for two test vectors");
  }
  k_fill_pattern<<<(unsigned)std::min<int64_t>(ceil_div(N, 256), 8 * kNumSMs), 256, 0, s>>>(c, N, dbl);
  // candidates: rows per warp x (CUDA-core chunk width | tensor-core pipeline depth)
  const bool cuda_core_ab = precision == HINQS_PREC_FP64 || precision == HINQS_PREC_FP32;
  std::vector<std::tuple<int, int, int>> cands;
  for (int r : {2, 4, 8}) {
    if (cuda_core_ab) {
      for (int ch : {16, 32}) cands.push_back({r, ch, 0});
    } else {
      // tensor-core pipeline depth 1 or 2 of the persistent kernel, or 3: the
      // tile-stationary warp-specialised kernel (BF16 operands only)
      for (int st : {1, 2, 3})
        if (st != 3 || precision != HINQS_PREC_FP32_BF16X3AB) cands.push_back({r, 0, st});
    }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 1e300;
  TuneVal bestv{0, 0, 0, 0.0};
  int rc = HINQS_OK;
  for (auto [r, ch, st] : cands) {
    la->tune_rows = lb->tune_rows = r;
    la->tune_ch = ch;
    la->tune_stages = st;
    if ((rc = sigma_launch(H, B, la, lb, c, sg, precision, s)) < 0) break;  // warm-up
    cudaEventRecord(e0, s);
    const int reps = 3;
    for (int k = 0; k < reps && rc >= 0; ++k) rc = sigma_launch(H, B, la, lb, c, sg, precision, s);
    if (rc < 0) break;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double t = ms / reps;
    if (t < best) {
      best = t;
      bestv = TuneVal{r, ch, st, t};
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(c, s);
  cudaFreeAsync(sg, s);
  if (rc < 0) return rc;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hinqs_autotune", __FILE__, __LINE__);
  la->tune_rows = lb->tune_rows = bestv.rows;
  la->tune_ch = bestv.ch;
  la->tune_stages = bestv.stages;
  if (best_ms) *best_ms = bestv.ms;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = bestv;
  return HINQS_OK;
}

// Rounds of sigma products.  Each running solve hands in one product per round
// (sigma) or leaves (leave); the thread whose hand-in completes a round launches it on
// the batch stream, after the ready events of every product's stream, and every
// product's stream then waits for the round's done event.
struct SigmaBatcher {
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;
  uint64_t round = 0;
  int round_rc = HINQS_OK;
  std::vector<SigmaReq> reqs;
  std::vector<cudaStream_t> streams;
  cudaStream_t bs = nullptr;
  cudaEvent_t done = nullptr;

  // with mu held
  void flush() {
    int rc = HINQS_OK;
    const int n = (int)reqs.size();
    if (n > 0) {
      rc = sigma_batch_launch(reqs.data(), n, bs);
      cudaError_t e = cudaEventRecord(done, bs);
      for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(streams[i], done, 0);
      if (rc >= 0 && e != cudaSuccess) rc = cuda_fail(e, "sigma batch round", __FILE__, __LINE__);
    }
    reqs.clear();
    streams.clear();
    round_rc = rc;
    ++round;
    cv.notify_all();
  }
};

int batcher_sigma(SigmaBatcher* b, const SigmaReq& r, cudaStream_t s, cudaEvent_t ready) {
  HQ_CUDA(cudaEventRecord(ready, s));
  std::unique_lock<std::mutex> lk(b->mu);
  HQ_CUDA(cudaStreamWaitEvent(b->bs, ready, 0));  // the round starts after this x is ready
  b->reqs.push_back(r);
  b->streams.push_back(s);
  const uint64_t my = b->round;
  if ((int)b->reqs.size() >= b->active) b->flush();
  else b->cv.wait(lk, [&] { return b->round != my; });
  return b->round_rc;
}

static void batcher_leave(SigmaBatcher* b) {
  std::lock_guard<std::mutex> lk(b->mu);
  --b->active;
  if (b->active > 0 && (int)b->reqs.size() >= b->active) b->flush();
}

}  // namespace hinqs

using namespace hinqs;

extern "C" int hinqs_autotune(const hinqs_ham* H, const hinqs_subspace* B, hinqs_links* la,
                              hinqs_links* lb, int precision, double* best_ms, void* stream) {
  HQ_TRY(check_triplet(H, B, la, lb, "hinqs_autotune"));
  if (precision < HINQS_PREC_FP64 || precision > HINQS_PREC_FP32_BF16C)
    return fail(HINQS_ERR_ARG, "hinqs_autotune: unknown precision %d", precision);
  return autotune_impl(H, B, la, lb, precision, best_ms, (cudaStream_t)stream);
}

extern "C" int hinqs_davidson_batch(int n_geom, const hinqs_ham* const* hams,
                                    const hinqs_subspace* const* subs, hinqs_links* const* las,
                                    hinqs_links* const* lbs, const double* const* guesses,
                                    const hinqs_davidson_opts* opts, int n_streams, int autotune,
                                    double* energies, double* const* c_outs,
                                    hinqs_davidson_info* infos, void* stream) {
  if (n_geom < 0 || (n_geom > 0 && (!hams || !subs || !las || !lbs || !c_outs || !energies)))
    return fail(HINQS_ERR_ARG, "hinqs_davidson_batch: NULL arrays");
  if (n_geom == 0) return HINQS_OK;
  for (int g = 0; g < n_geom; ++g) {
    HQ_TRY(check_triplet(hams[g], subs[g], las[g], lbs[g], "hinqs_davidson_batch"));
    if (!c_outs[g]) return fail(HINQS_ERR_ARG, "hinqs_davidson_batch: c_out[%d] is NULL", g);
  }
  hinqs_davidson_opts o;
  hinqs_davidson_default_opts(&o);
  if (opts) o = *opts;
  // the host trace arrays would be shared by the concurrent solves
  o.trace_cap = 0;
  o.trace_theta = o.trace_resid = o.trace_time = nullptr;
  o.trace_kind = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  // autotune the sigma the solve uses most (inner products of the mixed solver)
  if (autotune) {
    const int p = o.precision == HINQS_DAVIDSON_MIXED ? o.inner_precision : HINQS_PREC_FP64;
    for (int g = 0; g < n_geom; ++g) HQ_TRY(autotune_impl(hams[g], subs[g], las[g], lbs[g], p, nullptr, s));
  }
  // Lockstep (n_streams <= 0): the geometries below kBatchSoloN determinants hand their
  // sigma products to shared rounds (one thread and stream each); the larger ones, and
  // every geometry when n_streams > 0, go to worker streams, longest first.  Both sets
  // run at the same time.
  std::vector<int> small;
  std::vector<std::pair<double, int>> order;  // (cost, geometry) of the worker set
  for (int g = 0; g < n_geom; ++g) {
    const double Na = (double)subs[g]->Na, Nb = (double)subs[g]->Nb;
    if (n_streams <= 0 && subs[g]->Na * subs[g]->Nb < kBatchSoloN) {
      small.push_back(g);
      continue;
    }
    // cost ~ N * (links per alpha string + links per beta string + singles product)
    const double cost = Na * Nb *
                        ((double)las[g]->nnz / Na + (double)lbs[g]->nnz / Nb +
                         ((double)las[g]->nsingle / Na) * ((double)lbs[g]->nsingle / Nb + 1.0));
    order.push_back({cost, g});
  }
  std::sort(order.begin(), order.end(), [](auto& a, auto& b) { return a.first > b.first; });
  const int nw = order.empty() ? 0 : std::max(1, std::min(n_streams > 0 ? n_streams : 4,
                                                          (int)order.size()));
  const int ns = (int)small.size();
  // every stream starts after the caller's stream reaches this point
  cudaEvent_t start;
  HQ_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  HQ_CUDA(cudaEventRecord(start, s));
  std::vector<cudaStream_t> ws(nw), gs(ns);
  std::vector<cudaEvent_t> ready(ns);
  SigmaBatcher bat;
  bat.active = ns;
  auto make_stream = [&](cudaStream_t* st) -> int {
    HQ_CUDA(cudaStreamCreateWithFlags(st, cudaStreamNonBlocking));
    HQ_CUDA(cudaStreamWaitEvent(*st, start, 0));
    return HINQS_OK;
  };
  if (ns > 0) {
    HQ_TRY(make_stream(&bat.bs));
    HQ_CUDA(cudaEventCreateWithFlags(&bat.done, cudaEventDisableTiming));
  }
  for (int w = 0; w < nw; ++w) HQ_TRY(make_stream(&ws[w]));
  for (int k = 0; k < ns; ++k) {
    HQ_TRY(make_stream(&gs[k]));
    HQ_CUDA(cudaEventCreateWithFlags(&ready[k], cudaEventDisableTiming));
  }
  std::atomic<int> next{0};
  std::vector<int> status(n_geom, HINQS_OK);
  std::vector<std::string> msg(n_geom);
  std::vector<hinqs_davidson_info> inf(n_geom);
  int dev = 0;
  cudaGetDevice(&dev);
  auto solve = [&](int g, cudaStream_t st, SigmaBatcher* b, cudaEvent_t rdy) {
    double e = 0.0;
    status[g] = davidson_run(hams[g], subs[g], las[g], lbs[g], nullptr,
                             guesses ? guesses[g] : nullptr, &o, &e, c_outs[g], &inf[g],
                             (void*)st, "hinqs_davidson_batch", b, rdy);
    energies[g] = e;
    if (status[g] < 0) msg[g] = hinqs_last_error_message();
  };
  std::vector<std::thread> threads;
  for (int w = 0; w < nw; ++w)
    threads.emplace_back([&, w]() {
      cudaSetDevice(dev);
      for (int k; (k = next.fetch_add(1)) < (int)order.size();)
        solve(order[k].second, ws[w], nullptr, nullptr);
    });
  for (int k = 0; k < ns; ++k)
    threads.emplace_back([&, k]() {
      cudaSetDevice(dev);
      solve(small[k], gs[k], &bat, ready[k]);
      batcher_leave(&bat);
    });
  for (auto& t : threads) t.join();
  // the caller's stream continues after every stream
  auto join_stream = [&](cudaStream_t st) {
    cudaEvent_t done;
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    cudaEventRecord(done, st);
    cudaStreamWaitEvent(s, done, 0);
    cudaEventDestroy(done);
    cudaStreamDestroy(st);
  };
  for (int w = 0; w < nw; ++w) join_stream(ws[w]);
  for (int k = 0; k < ns; ++k) {
    join_stream(gs[k]);
    cudaEventDestroy(ready[k]);
  }
  if (ns > 0) {
    join_stream(bat.bs);
    cudaEventDestroy(bat.done);
  }
  cudaEventDestroy(start);
  int rc = HINQS_OK;
  for (int g = 0; g < n_geom; ++g) {
    if (infos) infos[g] = inf[g];
    if (status[g] < 0 && rc >= 0) {
      rc = status[g];
      set_error("hinqs_davidson_batch: geometry %d: %s", g, msg[g].c_str());
    } else if (status[g] > 0 && rc == HINQS_OK) {
      rc = status[g];
    }
  }
  return rc;
}
