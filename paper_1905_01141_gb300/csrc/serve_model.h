// serve_model.h -- the serving loop's host-side bookkeeping, free of CUDA:
// the rings that hold queued requests' LLRs and unpolled results, and the
// admission model that predicts when a subframe admitted now would finish.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <deque>

namespace crnt {

// Admission by predicted completion.  A TB admitted now finishes, on
// average, a + b X after its submission, where X is the expected decode
// work -- trellis steps times the iteration limit -- of every TB admitted
// and not yet finished, its own subframe's included: the work ahead of it
// drains at a rate 1/b, and a covers the launch, one decode and the
// collection.  (a, b) is refitted by least squares, with exponential
// forgetting, to the completions seen -- each TB gives one (X at its
// admission, latency) pair -- and held near prior values by a penalty that
// counts as a few pseudo-observations, so a cold start, or a load that
// leaves X nearly constant, keeps a sensible slope.  The residuals' spread
// sigma gives the margin: a subframe is refused when a + b X + z sigma
// passes the deadline, unless nothing at all is outstanding.  The fit is
// robust to stalls (TBs that waited for a one-time allocation, a descheduled
// thread): a latency above 8 deadlines is a stall, not queueing, and is left
// out; the others enter clipped to within max(4 d, 50 us) of the current
// prediction, d a moving mean of the absolute residuals over ~2000
// completions, so one outlier moves the fit by a bounded step while a
// lasting change (a slower device) widens d within a few thousand
// completions and is then followed; sigma stays at or below a sixth of the
// deadline (so that the margin alone never refuses everything); and the rate
// stays above 5e10 units/s (a full batch at the iteration limit drains
// ~1.2e11).  Forgetting counts the completions that entered the fit.
struct Admission {
  static constexpr double kA0 = 150.0;     // prior latency with nothing ahead (us)
  static constexpr double kB0 = 1.0e-5;    // prior us per unit of work (1e11 units/s)
  static constexpr double kBmin = 2.0e-6;  // at most 5e11 units/s (~4x a full decode)
  static constexpr double kBmax = 2.0e-5;  // at least 5e10 units/s
  static constexpr double kPrior = 16.0;   // weight of the prior, in observations
  static constexpr double kXs = 2.0e7;     // work scale at which the slope prior acts
  static constexpr double kMemory = 50000.0;  // TBs after which an observation's weight is 1/e
  static constexpr double kZ = 3.0;
  static constexpr double kMadMemory = 2000.0;  // completions in the residual scale d
  double sw = 0, sx = 0, sy = 0, sxx = 0, sxy = 0, syy = 0;
  double a = kA0, b = kB0, sigma = 50.0;
  double mad = 20.0;  // d: moving mean of |latency - a - b x| (us)
  double predict(double x) const { return a + b * x + kZ * sigma; }
  // a latency observation as it enters the fit (and the residual scale)
  double clip(double x, double y) {
    const double p = a + b * x, m = std::max(4.0 * mad, 50.0);
    mad += (std::abs(y - p) - mad) / kMadMemory;
    return std::min(p + m, std::max(p - m, y));
  }
  // One batch's completions, summed.
  struct Batch {
    double n = 0, w = 0, x = 0, y = 0, xx = 0, xy = 0, yy = 0;
  };
  // One completion: x the work ahead of it at admission, y its latency (us).
  void observe(Batch& bt, double x, double y, double deadline_us) {
    bt.n += 1;
    if (y > 8.0 * deadline_us) return;  // a stall: nothing to learn
    y = clip(x, y);
    bt.w += 1;
    bt.x += x;
    bt.y += y;
    bt.xx += x * x;
    bt.xy += x * y;
    bt.yy += y * y;
  }
  // Fold in one batch and refit.
  void update(const Batch& bt, double deadline_us) {
    const double f = std::exp(-bt.w / kMemory);
    sw = sw * f + bt.w;
    sx = sx * f + bt.x;
    sy = sy * f + bt.y;
    sxx = sxx * f + bt.xx;
    sxy = sxy * f + bt.xy;
    syy = syy * f + bt.yy;
    const double sigma_max = deadline_us / 6.0;
    const double ka = kPrior, kb = kPrior * kXs * kXs;
    const double m00 = sw + ka, m01 = sx, m11 = sxx + kb;
    const double v0 = sy + ka * kA0, v1 = sxy + kb * kB0;
    const double det = m00 * m11 - m01 * m01;
    if (!(det > 0)) return;
    a = std::min(2000.0, std::max(10.0, (v0 * m11 - m01 * v1) / det));
    b = std::min(kBmax, std::max(kBmin, (m00 * v1 - m01 * v0) / det));
    if (sw > 0) {
      const double sse = syy - 2 * a * sy - 2 * b * sxy + a * a * sw + 2 * a * b * sx +
                         b * b * sxx;
      sigma = std::min(sigma_max, std::max(10.0, std::sqrt(std::max(0.0, sse / sw))));
    }
  }
};

// Ring holding the LLRs of queued and running requests, released in
// allocation order.  Each allocation is contiguous.
struct Ring {
  size_t cap = 0, head = 0, tail = 0;
  struct A {
    size_t end;
    bool done;
  };
  std::deque<A> q;
  uint64_t first_seq = 0;  // sequence number of q.front()
  bool alloc(size_t n, size_t* off, uint64_t* seq) {
    if (q.empty()) head = tail = 0;
    if (head >= tail) {  // free space: [head, cap) and [0, tail)
      if (cap - head >= n) {
        *off = head;
      } else if (tail > n) {
        *off = 0;
      } else {
        return false;
      }
    } else if (tail - head > n) {  // free space: [head, tail)
      *off = head;
    } else {
      return false;
    }
    head = *off + n;
    *seq = first_seq + q.size();
    q.push_back(A{head, false});
    return true;
  }
  void release(uint64_t seq) {
    q[seq - first_seq].done = true;
    while (!q.empty() && q.front().done) {
      tail = q.front().end;
      q.pop_front();
      first_seq++;
    }
  }
};

}  // namespace crnt
