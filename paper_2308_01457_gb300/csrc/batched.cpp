// Batched workload: many scatterers of uneven size (the paper's concurrently processed
// sub-systems, Section V-D; here whole scatterers rather than combination-technique blocks).
//
// fosb_assemble_efie_batched: the regular pairs of every scatterer in one persistent launch
// that takes (scatterer, tile) work items from a device ticket, then one launch for all
// touching pairs and one for all right-hand sides.  The tile shape of the persistent launch
// (test triangles per tile, CTAs per SM of its register bound) is chosen by an autotuner: the first call
// for a batch signature with tune = 1 times each candidate on the batch itself and keeps
// the fastest for the rest of the process.
//
// fosb_solve_batched: a host scheduler over the scatterers.  Worker threads, each with its
// own non-blocking stream, take scatterers largest first (longest-processing-time order,
// which balances uneven sizes) and run the factorisation and the refined solve; the
// factorisations are released when every scatterer is done, because cudaFree synchronises
// the whole device and would serialise the workers.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "fosb_internal.h"

namespace fosb {
cudaError_t launch_efie_regular_ff_batched(const DevMesh* const* meshes, const double* ks, double* const* Z,
                                           const int64_t* ldz, int nmesh, int warps, int min_ctas,
                                           void* scratch, size_t scratch_bytes, cudaStream_t s);
size_t regular_ff_batched_scratch_bytes(int nmesh);
size_t batched_items_bytes(int nmesh);
cudaError_t launch_singular_rhs_batched(const DevMesh* const* meshes, const double* ks, double* const* Z,
                                        const int64_t* ldz, double* const* b, const int64_t* ldb,
                                        const double* const* inc, const int64_t* n_inc, int nmesh, int nss,
                                        void* d_items, cudaStream_t s);
fosb_status ensure_rules_for(int nss);

namespace {

// tile shape of the persistent regular-pair launch: test triangles per tile (warps) and the
// CTAs per SM its register allocation is bounded for (more CTAs, fewer registers per thread)
struct Shape {
  int warps, min_ctas;
};
constexpr Shape kCandidates[] = {{4, 5}, {4, 4}, {8, 2}, {8, 1}};

std::mutex g_tune_mu;
std::map<std::tuple<int, int64_t, int64_t, int64_t>, std::pair<Shape, double>> g_tuned;

}  // namespace
}  // namespace fosb

extern "C" {

fosb_status fosb_assemble_efie_batched(int64_t nbatch, const fosb_mesh* meshes, const double* k,
                                       const fosb_quad_opts* opts, void* const* Z, const int64_t* ldz,
                                       const double* const* inc, const int64_t* n_inc, void* const* b,
                                       const int64_t* ldb, int tune, fosb_batch_tuning* chosen, void* stream) {
  using namespace fosb;
  if (nbatch <= 0 || nbatch > (1 << 20) || !meshes || !k || !Z || !ldz)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: bad batch arguments");
  const int nss = opts && opts->n_ss > 0 ? opts->n_ss : 5;
  const int arith = opts ? opts->arith : FOSB_ASM_FF;
  if (nss > 12) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: n_ss must be in 1..12");
  if (arith != FOSB_ASM_FF && arith != FOSB_ASM_FP64)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: regular pairs in FOSB_ASM_FF or FOSB_ASM_FP64");
  const int n = int(nbatch);
  std::vector<const DevMesh*> dm(n);
  std::vector<double*> dZ(n), db(n);
  std::vector<const double*> dinc(n, nullptr);
  std::vector<int64_t> ninc(n, 0), ldb_v(n, 0);
  int64_t sum_nt = 0, sum_nt2 = 0, inc_total = 0;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i] || !Z[i]) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: NULL mesh or Z");
    const DevMesh& m = meshes[i]->d;
    if (!(k[i] > 0.0) || !std::isfinite(k[i]) || ldz[i] < m.ne)
      return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: bad k or ldz of item " + std::to_string(i));
    if (arith == FOSB_ASM_FF && k[i] * m.diameter >= ff_max_phase())
      return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: k * diameter of item " + std::to_string(i) +
                                            " exceeds the float-float phase range; use FOSB_ASM_FP64");
    dm[i] = &m;
    dZ[i] = static_cast<double*>(Z[i]);
    if (n_inc && n_inc[i] > 0) {
      if (!inc || !inc[i] || !b || !b[i] || !ldb || ldb[i] < n_inc[i])
        return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: bad incidence of item " + std::to_string(i));
      for (int64_t q = 0; q < 9 * n_inc[i]; ++q)
        if (!std::isfinite(inc[i][q])) return fail(FOSB_ERR_INVALID_ARG, "fosb_assemble_efie_batched: non-finite incidence");
      ninc[i] = n_inc[i];
      db[i] = static_cast<double*>(b[i]);
      ldb_v[i] = ldb[i];
      inc_total += 9 * n_inc[i];
    }
    sum_nt += m.nt;
    sum_nt2 += m.nt * m.nt;
  }
  FOSB_TRY(ensure_rules_for(nss));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  FOSB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // scratch: regular-pair items + ticket, singular/RHS items, the incidences
  const size_t reg_bytes = (regular_ff_batched_scratch_bytes(n) + 255) / 256 * 256;
  const size_t it_bytes = (batched_items_bytes(n) + 255) / 256 * 256;
  Scratch scr(s);
  FOSB_CUDA(scr.alloc(reg_bytes + it_bytes + sizeof(double) * std::max<int64_t>(inc_total, 1)));
  char* base = static_cast<char*>(scr.p);
  double* d_inc_all = reinterpret_cast<double*>(base + reg_bytes + it_bytes);
  {
    std::vector<double> h_inc(std::max<int64_t>(inc_total, 1));
    int64_t off = 0;
    for (int i = 0; i < n; ++i)
      if (ninc[i] > 0) {
        std::copy(inc[i], inc[i] + 9 * ninc[i], h_inc.begin() + off);
        dinc[i] = d_inc_all + off;
        off += 9 * ninc[i];
      }
    FOSB_CUDA(cudaMemcpyAsync(d_inc_all, h_inc.data(), sizeof(double) * h_inc.size(), cudaMemcpyHostToDevice, s));
    FOSB_CUDA(cudaStreamSynchronize(s));  // h_inc is released at the end of this scope
  }
  auto zero_all = [&]() -> cudaError_t {
    for (int i = 0; i < n; ++i) {
      const int64_t N = dm[i]->ne;
      cudaError_t e = cudaMemset2DAsync(dZ[i], ldz[i] * 16, 0, N * 16, N, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  Shape shape = kCandidates[0];
  double tuned_ms = 0.0;
  const auto key = std::make_tuple(dev, int64_t(n), sum_nt, sum_nt2);
  if (arith == FOSB_ASM_FF) {
    bool have = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto it = g_tuned.find(key);
      if (it != g_tuned.end()) {
        shape = it->second.first;
        tuned_ms = it->second.second;
        have = true;
      }
    }
    if (!have && tune) {
      cudaEvent_t e0, e1;
      FOSB_CUDA(cudaEventCreate(&e0));
      FOSB_CUDA(cudaEventCreate(&e1));
      double best = 1e300;
      cudaError_t err = cudaSuccess;
      for (const Shape& c : kCandidates) {
        if ((err = zero_all()) != cudaSuccess) break;
        cudaEventRecord(e0, s);
        err = launch_efie_regular_ff_batched(dm.data(), k, dZ.data(), ldz, n, c.warps, c.min_ctas, base, reg_bytes,
                                             s);
        cudaEventRecord(e1, s);
        if (err != cudaSuccess || (err = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          shape = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      FOSB_CUDA(err);
      tuned_ms = best;
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[key] = {shape, best};
    }
  }
  FOSB_CUDA(zero_all());
  for (int i = 0; i < n; ++i)
    if (ninc[i] > 0) FOSB_CUDA(cudaMemset2DAsync(db[i], ldb_v[i] * 16, 0, ninc[i] * 16, dm[i]->ne, s));
  if (arith == FOSB_ASM_FF) {
    FOSB_CUDA(launch_efie_regular_ff_batched(dm.data(), k, dZ.data(), ldz, n, shape.warps, shape.min_ctas, base,
                                             reg_bytes, s));
  } else {
    for (int i = 0; i < n; ++i) FOSB_CUDA(launch_assemble_regular(*dm[i], k[i], FOSB_ASM_FP64, dZ[i], ldz[i], s));
  }
  FOSB_CUDA(launch_singular_rhs_batched(dm.data(), k, dZ.data(), ldz, db.data(), ldb_v.data(), dinc.data(), ninc.data(),
                                        n, nss, base + reg_bytes, s));
  if (chosen) {
    chosen->warps = arith == FOSB_ASM_FF ? shape.warps : 0;
    chosen->ctas_per_sm = arith == FOSB_ASM_FF ? shape.min_ctas : 0;
    chosen->tuned_ms = tuned_ms;
  }
  return FOSB_OK;
}

fosb_status fosb_solve_batched(int64_t nbatch, const void* const* Z, const int64_t* n, const int64_t* ldz,
                               const void* const* B, const int64_t* nrhs, const int64_t* ldb, void* const* X,
                               const int64_t* ldx, int prec, const fosb_refine_opts* ropt, int workers,
                               fosb_solve_stats* stats, int* item_status, void* stream) {
  using namespace fosb;
  if (nbatch <= 0 || !Z || !n || !ldz || !B || !nrhs || !ldb || !X || !ldx)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_solve_batched: bad batch arguments");
  if (prec != FOSB_FP64 && prec != FOSB_MIXED)
    return fail(FOSB_ERR_INVALID_ARG, "fosb_solve_batched: prec must be FOSB_FP64 or FOSB_MIXED (complex128)");
  for (int64_t i = 0; i < nbatch; ++i)
    if (!Z[i] || !B[i] || !X[i] || n[i] <= 0 || ldz[i] < n[i] || nrhs[i] < 0 || ldb[i] < nrhs[i] || ldx[i] < nrhs[i])
      return fail(FOSB_ERR_INVALID_ARG, "fosb_solve_batched: bad arguments of item " + std::to_string(i));
  int dev = 0;
  FOSB_CUDA(cudaGetDevice(&dev));
  cudaStream_t caller = static_cast<cudaStream_t>(stream);
  cudaEvent_t ready;
  FOSB_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  FOSB_CUDA(cudaEventRecord(ready, caller));  // every item waits for the caller's earlier work
  // largest first
  std::vector<int64_t> order(nbatch);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return n[a] > n[b]; });
  const int nw = int(std::max<int64_t>(1, std::min<int64_t>(workers > 0 ? workers : 4, nbatch)));
  std::atomic<int64_t> next{0};
  std::vector<fosb_lu> lus(nbatch, nullptr);
  std::vector<int> st(nbatch, FOSB_OK);
  std::vector<std::string> msg(nbatch);
  std::vector<fosb_solve_stats> ss(nbatch, fosb_solve_stats{0, 0.0});
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t ws = nullptr;
    if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess || cudaStreamWaitEvent(ws, ready, 0)) {
      for (int64_t q; (q = next.fetch_add(1)) < nbatch;) {
        st[order[q]] = FOSB_ERR_CUDA;
        msg[order[q]] = "fosb_solve_batched: worker stream";
      }
      if (ws) cudaStreamDestroy(ws);
      return;
    }
    for (int64_t q; (q = next.fetch_add(1)) < nbatch;) {
      const int64_t i = order[q];
      fosb_status r = fosb_factor(Z[i], n[i], ldz[i], prec, &lus[i], ws);
      if (r == FOSB_OK)
        r = fosb_solve(lus[i], 'N', B[i], nrhs[i], ldb[i], X[i], ldx[i], ropt, &ss[i], ws);
      st[i] = r;
      if (r != FOSB_OK) msg[i] = fosb_last_error();
    }
    cudaStreamSynchronize(ws);
    cudaStreamDestroy(ws);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  cudaEventDestroy(ready);
  for (auto* lu : lus)
    if (lu) fosb_lu_destroy(lu);
  fosb_status first = FOSB_OK;
  std::string first_msg;
  for (int64_t i = 0; i < nbatch; ++i) {
    if (stats) stats[i] = ss[i];
    if (item_status) item_status[i] = st[i];
    if (st[i] != FOSB_OK && first == FOSB_OK) {
      first = st[i];
      first_msg = "item " + std::to_string(i) + ": " + msg[i];
    }
  }
  if (first != FOSB_OK) return fail(first, first_msg);
  return FOSB_OK;
}

}  // extern "C"
