// Checks of the serving loop's host-side bookkeeping (serve_model.h): the
// ring allocator and the admission model.  Built and run by
// tests/test_serve_model.py; prints one line per check and exits non-zero on
// the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>

#include "serve_model.h"

using crnt::Admission;
using crnt::Ring;

static int fails = 0;
static void check(bool ok, const char* what) {
  std::printf("%s %s\n", ok ? "ok" : "FAIL", what);
  if (!ok) fails++;
}

static void ring_checks() {
  Ring r;
  r.cap = 100;
  size_t o[4];
  uint64_t q[4];
  check(r.alloc(30, &o[0], &q[0]) && o[0] == 0, "ring: first allocation at 0");
  check(r.alloc(30, &o[1], &q[1]) && o[1] == 30, "ring: second follows");
  check(r.alloc(30, &o[2], &q[2]) && o[2] == 60, "ring: third follows");
  size_t x;
  uint64_t qx;
  check(!r.alloc(20, &x, &qx), "ring: no room at the end and none before the oldest");
  r.release(q[1]);  // out of order: the oldest still holds its bytes
  check(!r.alloc(20, &x, &qx), "ring: an out-of-order release frees nothing yet");
  r.release(q[0]);  // now the first two are free
  check(r.alloc(20, &o[3], &q[3]) && o[3] == 0, "ring: wraps to the start once the oldest is free");
  check(!r.alloc(40, &x, &qx) , "ring: the wrapped region stops short of the oldest");
  r.release(q[2]);
  r.release(q[3]);
  check(r.alloc(100, &x, &qx) && x == 0, "ring: empty again, the whole ring");
}

// Latencies y = a + b x + noise for work x ahead, in batches of 16.
static void feed(Admission& m, std::mt19937_64& g, int batches, double a, double b, double sd,
                 double deadline) {
  std::uniform_real_distribution<double> ux(0.0, 6.0e7);
  std::normal_distribution<double> nz(0.0, sd);
  for (int k = 0; k < batches; k++) {
    Admission::Batch bt;
    for (int i = 0; i < 16; i++) {
      const double x = ux(g);
      m.observe(bt, x, a + b * x + nz(g), deadline);
    }
    m.update(bt, deadline);
  }
}

static void admission_checks() {
  const double D = 1000.0;
  std::mt19937_64 g(7);
  Admission m;
  feed(m, g, 3000, 120.0, 1.2e-5, 20.0, D);
  check(std::abs(m.a - 120.0) < 6.0, "admission: intercept recovered");
  check(std::abs(m.b - 1.2e-5) < 0.06 * 1.2e-5, "admission: rate recovered");
  check(m.sigma > 14.0 && m.sigma < 26.0, "admission: spread recovered");
  const double p0 = m.predict(3.0e7);
  // a stall (latency above 8 deadlines) is left out
  Admission::Batch st;
  for (int i = 0; i < 16; i++) m.observe(st, 1.0e6, 50000.0, D);
  const double a0 = m.a, b0 = m.b, s0 = m.sigma;
  m.update(st, D);
  check(st.w == 0 && std::abs(m.a - a0) < 1e-6 && std::abs(m.b - b0) < 1e-12 &&
            std::abs(m.sigma - s0) < 1e-6,
        "admission: a stall leaves the fit as it was");
  // one batch of 3 ms outliers (below the stall bound): a bounded step
  Admission::Batch ob;
  for (int i = 0; i < 16; i++) m.observe(ob, 1.0e6, 3000.0, D);
  m.update(ob, D);
  check(m.sigma <= 2.0 * s0 + 1e-9 && std::abs(m.predict(3.0e7) - p0) < 100.0,
        "admission: one outlier batch moves the prediction by a bounded step");
  // a lasting change (the device twice as slow) is followed
  feed(m, g, 3000, 120.0, 2.4e-5, 20.0, D);
  check(m.b > 1.8e-5, "admission: a lasting slowdown is followed");
  // the spread never exceeds a sixth of the deadline
  Admission w;
  feed(w, g, 500, 150.0, 1.0e-5, 2000.0, D);
  check(w.sigma <= D / 6.0 + 1e-9, "admission: spread capped at a sixth of the deadline");
  // a cold start that begins with stalled batches stays usable: after normal
  // traffic a light load is admitted (predicted well inside the deadline)
  Admission c;
  for (int k = 0; k < 4; k++) {
    Admission::Batch sb;
    for (int i = 0; i < 8; i++) c.observe(sb, 1.0e6, 5000.0 + 1000.0 * k, D);
    c.update(sb, D);
  }
  feed(c, g, 200, 150.0, 1.0e-5, 20.0, D);
  check(c.predict(2.0e6) < 0.5 * D, "admission: a startup stall does not outlast the start");
}

int main() {
  ring_checks();
  admission_checks();
  std::printf("%d failures\n", fails);
  return fails ? 1 : 0;
}
