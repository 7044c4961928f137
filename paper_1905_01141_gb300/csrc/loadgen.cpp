// loadgen.cpp -- open-loop cell load for the serving loop, a client of the
// public C ABI only (crnt_submit / crnt_poll).
//
// Every cell sends one subframe (its UEs' TBs) per 1 ms period, at a random
// phase plus uniform jitter, from native submitter threads that follow the
// arrival times; a poller thread collects results.  Latency of a TB = its
// completion time (the library's t_done_ns, steady clock) minus its
// scheduled arrival.  A fraction of TBs are HARQ retransmissions of the same
// (cell, UE, process) with the redundancy version cycling 2, 3, 1, 0.
//
// Input file (written by the caller): uint32 n, then n crnt_tb_params, then
// n int64 LLR offsets, then the LLR bytes.  TB u of cell c is entry
// (c * ues + u) mod n.  Output: one JSON object per cell count on stdout.
//
// usage: crnt_loadgen [--tune TABLE] [--purge] [--poisson] [--admit-by-count] [--threads T]
//                     FILE UES SECONDS RETX_FRACTION SEED CELLS...
// TABLE: a window-count table (188 numbers) installed with crnt_tune_set,
// optionally followed by a radix table (188 numbers, crnt_tune_radix_set)
// and a CTA-shape table (188 numbers, crnt_tune_shape_set);
// --purge: every TB asks for purge on failure (CRNT_F_PURGE);
// --poisson: exponential inter-arrival times of mean 1 ms per cell instead of
// the 1 ms period with jitter; --admit-by-count: the library admits by its
// in-flight and memory limits only, not by predicted completion;
// --threads T: submitter threads, cells dealt round-robin (default 4; each
// copies its cells' LLRs in crnt_submit).
// Each output line also splits the latency into its parts (p50, p99 in us):
// scheduled arrival -> submit call, submit -> launch of the TB's batch,
// launch -> result collected; and gives the library's serving counters over
// the point (crnt_serve_stats_get): offered and admitted TBs, subframes
// refused for their predicted completion, batches, the serving worker's time
// shares, the submitting threads' copy time in cores, the admission model.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <queue>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/crnt.h"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

// SplitMix64 (public definition): the phases, jitter and retransmission draws
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unit(uint64_t& s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

struct Point {
  int cells = 0;
  long tbs = 0, subframes = 0, refused = 0, errors = 0;
  double p50 = 0, p99 = 0, miss = 0, gbit = 0;
  // latency parts (p50, p99 in us): scheduled arrival -> submit call,
  // submit -> launch of its batch, launch -> result collected
  double part[3][2] = {};
  crnt_serve_stats st{};  // the library's counters over the point
};

double pct(std::vector<double>& v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  return v[std::min(v.size() - 1, (size_t)(q * (double)v.size()))];
}

Point run_point(crnt_ctx* ctx, const std::vector<crnt_tb_params>& par,
                const std::vector<const int8_t*>& ptr, int ues, int cells, double seconds,
                double retx, uint64_t seed, uint32_t extra_flags, bool poisson, int nthreads) {
  const int n = (int)par.size();
  uint64_t rs = seed * 1000003ull + (uint64_t)cells;
  std::vector<double> phase(cells);
  for (int c = 0; c < cells; c++) phase[c] = unit(rs) * 1e6;
  std::mutex mu;
  // ticket -> (arrival, A); results that arrive before their ticket is
  // registered wait in `early` (ticket -> (done time, status))
  std::unordered_map<uint64_t, std::pair<int64_t, uint32_t>> pending;
  std::unordered_map<uint64_t, crnt_tb_result> early;
  std::vector<double> lat, parts[3];
  std::atomic<int> submitting{nthreads};
  long n_bits = 0, errors = 0;
  const int64_t t0 = now_ns() + 2000000;
  const int64_t t_end = t0 + (int64_t)(seconds * 1e9);
  auto record = [&](int64_t arrival, uint32_t A, const crnt_tb_result& r) {
    if (r.status != CRNT_OK) errors++;
    lat.push_back((double)((int64_t)r.t_done_ns - arrival) / 1e3);
    parts[0].push_back((double)((int64_t)r.t_submit_ns - arrival) / 1e3);
    parts[1].push_back((double)((int64_t)r.t_start_ns - (int64_t)r.t_submit_ns) / 1e3);
    parts[2].push_back((double)((int64_t)r.t_done_ns - (int64_t)r.t_start_ns) / 1e3);
    n_bits += A;
  };
  crnt_serve_stats st0;
  crnt_serve_stats_get(ctx, &st0);
  // poller
  std::thread poller([&] {
    std::vector<crnt_tb_result> res(4096);
    std::vector<const uint8_t*> bits(4096);
    for (;;) {
      const int k = crnt_poll(ctx, res.data(), bits.data(), 4096, 1000);
      if (k < 0) break;
      std::lock_guard<std::mutex> lk(mu);
      for (int i = 0; i < k; i++) {
        auto it = pending.find(res[i].ticket);
        if (it == pending.end()) {
          early[res[i].ticket] = res[i];
          continue;
        }
        record(it->second.first, it->second.second, res[i]);
        pending.erase(it);
      }
      if (submitting.load() == 0 && pending.empty() && early.empty()) break;
      if (now_ns() > t_end + 5000000000ll) break;
    }
  });
  // submitters: thread h serves the cells c with c mod nthreads == h, each
  // in arrival-time order (several threads, as several fronthaul links
  // would, so that the host-side copies of the LLRs are not one core's work)
  std::atomic<long> subframes{0}, refused{0};
  auto submitter = [&](int h) {
    uint64_t rh = seed * 7919ull + (uint64_t)cells * 131ull + (uint64_t)h;
    using Ev = std::pair<int64_t, int>;  // (arrival, cell)
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> q;
    std::vector<int> sf(cells, 0);
    for (int c = h; c < cells; c += nthreads) q.push(Ev{t0 + (int64_t)phase[c], c});
    std::vector<crnt_tb_params> tb(ues);
    std::vector<const int8_t*> lp(ues);
    std::vector<uint64_t> tk(ues);
    while (!q.empty()) {
      const Ev ev = q.top();
      q.pop();
      if (ev.first >= t_end) continue;
      while (now_ns() < ev.first) {
      }
      const int c = ev.second;
      const int pid = sf[c] % 8;
      for (int u = 0; u < ues; u++) {
        const int e = (c * ues + u) % n;
        tb[u] = par[e];
        lp[u] = ptr[e];
        tb[u].cell = (uint32_t)c;
        tb[u].ue = (uint32_t)u;
        tb[u].harq_pid = (uint32_t)pid;
        tb[u].flags = CRNT_F_HARQ | extra_flags;
        const bool rt = sf[c] >= 8 && unit(rh) < retx;
        static const uint8_t rv_cycle[4] = {2, 3, 1, 0};
        tb[u].new_data = rt ? 0 : 1;
        tb[u].rv = rt ? rv_cycle[(sf[c] / 8) % 4] : 0;
      }
      const int rc = crnt_submit(ctx, tb.data(), lp.data(), (uint32_t)ues, tk.data());
      if (rc == CRNT_OK) {
        std::lock_guard<std::mutex> lk(mu);
        for (int u = 0; u < ues; u++) {
          auto it = early.find(tk[u]);
          if (it != early.end()) {
            record(ev.first, tb[u].A, it->second);
            early.erase(it);
          } else {
            pending[tk[u]] = {ev.first, tb[u].A};
          }
        }
      } else {
        refused++;
      }
      subframes++;
      sf[c]++;
      if (poisson) {
        const double gap = -std::log(1.0 - unit(rh)) * 1e6;  // exponential, mean 1 ms
        q.push(Ev{ev.first + (int64_t)gap, c});
      } else {
        const double jit = (unit(rh) - 0.5) * 400000.0;
        q.push(Ev{t0 + (int64_t)sf[c] * 1000000 + (int64_t)(phase[c] + jit), c});
      }
    }
    submitting--;
  };
  std::vector<std::thread> subs;
  for (int h = 0; h < nthreads; h++) subs.emplace_back(submitter, h);
  for (auto& th : subs) th.join();
  poller.join();
  Point p;
  p.cells = cells;
  p.subframes = subframes.load();
  p.refused = refused.load();
  p.errors = errors;
  std::sort(lat.begin(), lat.end());
  p.tbs = (long)lat.size();
  if (!lat.empty()) {
    p.p50 = lat[lat.size() / 2];
    p.p99 = lat[std::min(lat.size() - 1, (size_t)(0.99 * (double)lat.size()))];
    long miss = 0;
    for (double x : lat) miss += x > 1000.0;
    p.miss = (double)miss / (double)lat.size();
  }
  p.gbit = (double)n_bits / seconds / 1e9;
  for (int k = 0; k < 3; k++) {
    p.part[k][1] = pct(parts[k], 0.99);
    p.part[k][0] = pct(parts[k], 0.5);
  }
  crnt_serve_stats st1;
  crnt_serve_stats_get(ctx, &st1);
  p.st = st1;  // counters over the point; the model fields are its state at the end
  p.st.submit_calls -= st0.submit_calls;
  p.st.refused_calls -= st0.refused_calls;
  p.st.refused_deadline -= st0.refused_deadline;
  p.st.offered_tbs -= st0.offered_tbs;
  p.st.admitted_tbs -= st0.admitted_tbs;
  p.st.done_tbs -= st0.done_tbs;
  p.st.late_tbs -= st0.late_tbs;
  p.st.batches -= st0.batches;
  p.st.worker_plan_ns -= st0.worker_plan_ns;
  p.st.worker_launch_ns -= st0.worker_launch_ns;
  p.st.worker_harvest_ns -= st0.worker_harvest_ns;
  p.st.worker_ns -= st0.worker_ns;
  p.st.submit_copy_ns -= st0.submit_copy_ns;
  return p;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc > 2 && strcmp(argv[1], "--tune") == 0) {
    FILE* t = fopen(argv[2], "r");
    if (!t) return 2;
    uint8_t table[CRNT_NUM_K], radix[CRNT_NUM_K];
    for (int i = 0; i < CRNT_NUM_K; i++) {
      int v = 0;
      if (fscanf(t, "%d", &v) != 1) return 2;
      table[i] = (uint8_t)v;
    }
    int nr = 0;  // an optional radix table follows
    for (; nr < CRNT_NUM_K; nr++) {
      int v = 0;
      if (fscanf(t, "%d", &v) != 1) break;
      radix[nr] = (uint8_t)v;
    }
    uint8_t shape[CRNT_NUM_K];
    int ns = 0;  // and an optional CTA-shape table
    for (; nr == CRNT_NUM_K && ns < CRNT_NUM_K; ns++) {
      int v = 0;
      if (fscanf(t, "%d", &v) != 1) break;
      shape[ns] = (uint8_t)v;
    }
    fclose(t);
    if (crnt_tune_set(table, CRNT_NUM_K) != CRNT_OK) return 2;
    if (nr == CRNT_NUM_K && crnt_tune_radix_set(radix, CRNT_NUM_K) != CRNT_OK) return 2;
    if (ns == CRNT_NUM_K && crnt_tune_shape_set(shape, CRNT_NUM_K) != CRNT_OK) return 2;
    argv += 2;
    argc -= 2;
  }
  uint32_t extra_flags = 0, admission = 0;
  bool poisson = false;
  int nthreads = 4;
  for (;;) {
    if (argc > 1 && strcmp(argv[1], "--purge") == 0) {
      extra_flags = CRNT_F_PURGE;
    } else if (argc > 1 && strcmp(argv[1], "--poisson") == 0) {
      poisson = true;
    } else if (argc > 1 && strcmp(argv[1], "--admit-by-count") == 0) {
      admission = 1;
    } else if (argc > 2 && strcmp(argv[1], "--threads") == 0) {
      nthreads = std::max(1, std::min(64, atoi(argv[2])));
      argv += 1;
      argc -= 1;
    } else {
      break;
    }
    argv += 1;
    argc -= 1;
  }
  if (argc < 7) {
    fprintf(stderr,
            "usage: crnt_loadgen [--tune TABLE] [--purge] [--poisson] [--admit-by-count] "
            "[--threads T] FILE UES SECONDS RETX SEED CELLS...\n");
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  uint32_t n = 0;
  if (fread(&n, 4, 1, f) != 1 || n == 0) return 2;
  std::vector<crnt_tb_params> par(n);
  std::vector<int64_t> off(n);
  if (fread(par.data(), sizeof(crnt_tb_params), n, f) != n || fread(off.data(), 8, n, f) != n)
    return 2;
  std::vector<int8_t> blob;
  int8_t buf[1 << 16];
  size_t k;
  while ((k = fread(buf, 1, sizeof buf, f)) > 0) blob.insert(blob.end(), buf, buf + k);
  fclose(f);
  std::vector<const int8_t*> ptr(n);
  for (uint32_t i = 0; i < n; i++) ptr[i] = blob.data() + off[i];
  const int ues = atoi(argv[2]);
  const double seconds = atof(argv[3]), retx = atof(argv[4]);
  const uint64_t seed = strtoull(argv[5], nullptr, 10);
  int max_cells = 0;
  for (int a = 6; a < argc; a++) max_cells = std::max(max_cells, atoi(argv[a]));
  crnt_config cfg;
  memset(&cfg, 0, sizeof cfg);
  cfg.harq_slots = (uint32_t)std::max(4096, max_cells * ues * 8);
  cfg.max_inflight = 65536;
  cfg.admission = admission;
  crnt_ctx* ctx = nullptr;
  if (crnt_create(&ctx, &cfg) != CRNT_OK) return 3;
  // warm-up passes (not reported): the serving loop's buffers, the HARQ
  // arena and every kernel the mix uses come up here
  for (int w = 0; w < 2; w++)
    run_point(ctx, par, ptr, ues, std::min(16 << w, max_cells), 0.3, retx, seed + 1 + w,
              extra_flags, poisson, nthreads);
  for (int a = 6; a < argc; a++) {
    const int cells = atoi(argv[a]);
    const Point p =
        run_point(ctx, par, ptr, ues, cells, seconds, retx, seed, extra_flags, poisson, nthreads);
    const crnt_serve_stats& s = p.st;
    const double wall = s.worker_ns ? (double)s.worker_ns : 1.0;
    printf("{\"cells\": %d, \"tbs\": %ld, \"subframes\": %ld, \"refused_subframes\": %ld, "
           "\"errors\": %ld, \"p50_us\": %.1f, \"p99_us\": %.1f, \"deadline_miss\": %.6f, "
           "\"gbit_s\": %.4f, \"submit_lag_us\": [%.1f, %.1f], \"queue_us\": [%.1f, %.1f], "
           "\"device_us\": [%.1f, %.1f], \"offered_tbs\": %llu, \"admitted_tbs\": %llu, "
           "\"refused_deadline\": %llu, \"batches\": %llu, \"worker_busy\": "
           "{\"plan\": %.3f, \"launch\": %.3f, \"harvest\": %.3f}, "
           "\"copy_cores\": %.3f, \"model\": {\"a_us\": %.1f, \"rate\": %.1f, "
           "\"sigma_us\": %.1f}}\n",
           p.cells, p.tbs, p.subframes, p.refused, p.errors, p.p50, p.p99, p.miss, p.gbit,
           p.part[0][0], p.part[0][1], p.part[1][0], p.part[1][1], p.part[2][0], p.part[2][1],
           (unsigned long long)s.offered_tbs, (unsigned long long)s.admitted_tbs,
           (unsigned long long)s.refused_deadline, (unsigned long long)s.batches,
           s.worker_plan_ns / wall, s.worker_launch_ns / wall, s.worker_harvest_ns / wall,
           s.submit_copy_ns / wall, s.model_a_us, s.model_rate, s.model_sigma_us);
    fflush(stdout);
    // far past saturation: most subframes late by more than 20 ms at p99 (an
    // isolated host stall can push p99 up at light load without that)
    if (p.p99 > 20000.0 && p.miss > 0.5) break;
  }
  crnt_destroy(ctx);
  return 0;
}
