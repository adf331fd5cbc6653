// Expectation values of local terms and their sum (Sec. V: the energy is
// the sum over the Hamiltonian's terms of <Psi|h_t|Psi> / <Psi|Psi>, each
// term and the norm contracted as a closed network; the cluster
// approximation of Fig. 4b gives every term its own pair of networks).
//
// ftn_energy_reduce turns contracted network values, kept as (mantissa,
// natural-log scale) pairs, into per-term ratios and FP64 sums; it is host
// arithmetic on a few doubles per term and touches no device.  ftn_energy
// contracts the networks first: contexts on their own streams each run on
// one host thread and take networks (or lock-step batches of networks) from
// a shared counter, so independent contractions overlap on the GPU; results
// land in fixed slots and the sums run in term order, so the values do not
// depend on the schedule.
#include <atomic>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.h"

using namespace ftn;

namespace {

ftn_status check_terms(int count, int n_terms, const int32_t* num, const int32_t* den, int n_groups,
                       const int32_t* group_end) {
  if (count < 0 || n_terms < 0 || n_groups < 0) return set_error(FTN_EINVAL, "negative count");
  if (n_terms > 0 && (!num || !den)) return set_error(FTN_EINVAL, "null term index array");
  if (n_groups > 0 && !group_end) return set_error(FTN_EINVAL, "null group_end");
  for (int t = 0; t < n_terms; ++t)
    if (num[t] < 0 || num[t] >= count || den[t] < 0 || den[t] >= count)
      return set_error(FTN_EINVAL, "term network index out of range");
  int prev = 0;
  for (int g = 0; g < n_groups; ++g) {
    if (group_end[g] < prev || group_end[g] > n_terms)
      return set_error(FTN_EINVAL, "group_end must be non-decreasing and at most n_terms");
    prev = group_end[g];
  }
  return FTN_OK;
}

}  // namespace

extern "C" {

ftn_status ftn_energy_reduce(int count, const double* mantissa, const double* log_scale, int n_terms,
                             const int32_t* num, const int32_t* den, int n_groups, const int32_t* group_end,
                             double* ratios, double* energies) {
  FTN_TRY(check_terms(count, n_terms, num, den, n_groups, group_end));
  if (count > 0 && (!mantissa || !log_scale)) return set_error(FTN_EINVAL, "null network values");
  if (n_groups > 0 && !energies) return set_error(FTN_EINVAL, "null energies");
  std::vector<double> r(n_terms);
  for (int t = 0; t < n_terms; ++t) {
    const double md = mantissa[den[t]];
    if (!(md != 0.0) || !std::isfinite(md) || !std::isfinite(log_scale[den[t]]))
      return set_error(FTN_EINVAL, "a denominator network has a zero or non-finite value");
    r[t] = mantissa[num[t]] / md * std::exp(log_scale[num[t]] - log_scale[den[t]]);
  }
  int t0 = 0;
  for (int g = 0; g < n_groups; ++g) {
    double s = 0.0;
    for (int t = t0; t < group_end[g]; ++t) s += r[t];
    energies[g] = s;
    t0 = group_end[g];
  }
  if (ratios)
    for (int t = 0; t < n_terms; ++t) ratios[t] = r[t];
  return FTN_OK;
}

ftn_status ftn_energy(int n_ctx, const ftn_ctx* ctxs, int count, const ftn_network* nets, const ftn_tree* trees,
                      ftn_prec prec, int batch, double* mantissa, double* log_scale, int n_terms, const int32_t* num,
                      const int32_t* den, int n_groups, const int32_t* group_end, double* ratios, double* energies) {
  if (n_ctx < 1 || !ctxs) return set_error(FTN_EINVAL, "need at least one context");
  for (int i = 0; i < n_ctx; ++i)
    if (!ctxs[i]) return set_error(FTN_EINVAL, "null context");
  if (count > 0 && (!nets || !trees)) return set_error(FTN_EINVAL, "null network or tree array");
  if (batch < 0) return set_error(FTN_EINVAL, "batch must be >= 0");
  FTN_TRY(check_terms(count, n_terms, num, den, n_groups, group_end));
  if (n_groups > 0 && !energies) return set_error(FTN_EINVAL, "null energies");
  std::vector<double> m(count), l(count);
  // jobs: [first network, end) ranges; batch 0 = one ftn_contract per network
  std::vector<std::pair<int, int>> jobs;
  const int step = batch > 0 ? batch : 1;
  for (int i = 0; i < count; i += step) jobs.push_back({i, std::min(count, i + step)});
  // the inputs may come from work queued on the first context's stream
  FTN_CUDA(cudaStreamSynchronize(ctxs[0]->stream));
  std::atomic<size_t> next{0};
  std::atomic<bool> failed{false};
  std::mutex mu;
  ftn_status first = FTN_OK;
  std::string msg;
  auto worker = [&](ftn_ctx c) {
    if (cudaSetDevice(c->device) != cudaSuccess) {
      std::lock_guard<std::mutex> g(mu);
      if (first == FTN_OK) first = FTN_ECUDA, msg = "cudaSetDevice failed in an ftn_energy worker";
      failed = true;
      return;
    }
    while (!failed) {
      const size_t j = next.fetch_add(1);
      if (j >= jobs.size()) return;
      const int a = jobs[j].first, b = jobs[j].second;
      const ftn_status st = batch > 0 ? ftn_contract_batch(c, b - a, nets + a, trees + a, prec, &m[a], &l[a])
                                      : ftn_contract(c, nets + a, trees + a, prec, &m[a], &l[a]);
      if (st != FTN_OK) {
        std::lock_guard<std::mutex> g(mu);
        if (first == FTN_OK) first = st, msg = ftn_last_error();
        failed = true;
      }
    }
  };
  if (n_ctx == 1 || jobs.size() <= 1) {
    worker(ctxs[0]);
  } else {
    std::vector<std::thread> th;
    for (int i = 0; i < n_ctx; ++i) th.emplace_back(worker, ctxs[i]);
    for (auto& t : th) t.join();
  }
  if (first != FTN_OK) return set_error(first, msg);
  if (mantissa)
    for (int i = 0; i < count; ++i) mantissa[i] = m[i];
  if (log_scale)
    for (int i = 0; i < count; ++i) log_scale[i] = l[i];
  return ftn_energy_reduce(count, m.data(), l.data(), n_terms, num, den, n_groups, group_end, ratios, energies);
}

}  // extern "C"
