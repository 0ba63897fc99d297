// When a run is steady: the test on the hot-wall Nusselt history and the drivers that step a
// cavity or a batch until it holds. The paper reports steady states only (Sec. 3: the hot-wall
// Nu of Figs 3, 5-7) and does not say when a run counts as steady; the reading here: "the
// distance to the steady hot-wall Nu is at most tol |Nu|", judged on several lags of the
// history so that a fast mode that has settled does not hide a slow one still moving Nu (the
// particle component's migration, 1e5-1e6 steps).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "mclbm_internal.h"

namespace {

constexpr double kFloorPerLag = 2e-7;  // FP32 round-off floor of one check's change, per lag
constexpr double kRatioSpread = 0.05;  // the four ratios of a geometric tail agree this well
constexpr double kRatioMax = 0.99;     // slower tails are not extrapolated
constexpr int kMaxLags = 8;
const int32_t kDefaultLags[2] = {1, 32};

// Six values p[0..5] (latest first, equally spaced): steady when (a) the last two changes are at
// the round-off floor, (b) Nu oscillates (two or more sign flips among the five changes) within
// half the tolerance, or (c) the changes shrink geometrically with one sign and a consistent
// ratio r, and the rest of that series, |d_0| r / (1 - r), is within tol |Nu|.
bool tail_ok(const double* p, double tol, double floor) {
  const double nu = p[0];
  double d[5];
  for (int k = 0; k < 5; ++k) d[k] = p[k] - p[k + 1];
  const double lim = floor * std::fabs(nu);
  if (std::fabs(d[0]) <= lim && std::fabs(d[1]) <= lim) return true;
  int flips = 0;
  for (int k = 0; k < 4; ++k)
    if (d[k] * d[k + 1] < 0.0) ++flips;
  double lo = p[0], hi = p[0];
  for (int k = 1; k < 6; ++k) {
    lo = std::fmin(lo, p[k]);
    hi = std::fmax(hi, p[k]);
  }
  if (flips >= 2 && hi - lo <= 0.5 * tol * std::fabs(nu)) return true;
  for (int k = 1; k < 5; ++k)
    if (d[k] == 0.0) return false;
  double r[4], rmin = 0.0, rmax = 0.0;
  for (int k = 0; k < 4; ++k) {
    r[k] = d[k] / d[k + 1];
    if (!(r[k] >= 0.0 && r[k] < kRatioMax)) return false;
    rmin = k ? std::fmin(rmin, r[k]) : r[k];
    rmax = k ? std::fmax(rmax, r[k]) : r[k];
  }
  if (rmax - rmin > kRatioSpread) return false;
  return std::fabs(d[0]) * rmax / (1.0 - rmax) <= tol * std::fabs(nu);
}

bool args_ok(double tol, const int32_t* lags, int n_lags) {
  if (!(tol > 0.0) || n_lags < 1 || n_lags > kMaxLags || !lags) return false;
  for (int l = 0; l < n_lags; ++l)
    if (lags[l] < 1 || lags[l] > (1 << 20)) return false;
  return true;
}

int steady(const double* h, int64_t n, double tol, const int32_t* lags, int n_lags) {
  int64_t need = 1;
  for (int l = 0; l < n_lags; ++l) need = std::max<int64_t>(need, 5 * (int64_t)lags[l] + 1);
  if (n < need) return 0;
  for (int l = 0; l < n_lags; ++l) {
    double p[6];
    for (int k = 0; k < 6; ++k) p[k] = h[n - 1 - (int64_t)k * lags[l]];
    if (!tail_ok(p, tol, kFloorPerLag * lags[l])) return 0;
  }
  return 1;
}

}  // namespace

extern "C" {

int mclbm_steady_nu_reached(const double* nu_hist, int64_t n, double tol, const int32_t* lags,
                            int n_lags) {
  if (!lags) {
    lags = kDefaultLags;
    n_lags = 2;
  }
  if (n < 0 || (n > 0 && !nu_hist) || !args_ok(tol, lags, n_lags)) return MCLBM_EINVAL;
  return steady(nu_hist, n, tol, lags, n_lags);
}

int mclbm_run_to_steady(mclbm_t* h, double tol, int64_t check_every, int64_t max_steps,
                        const int32_t* lags, int n_lags, int64_t* steps, double* nu_hot,
                        double* nu_cold, int* converged) {
  if (!lags) {
    lags = kDefaultLags;
    n_lags = 2;
  }
  if (!h || check_every < 1 || max_steps < 0 || !args_ok(tol, lags, n_lags)) return MCLBM_EINVAL;
  std::vector<double> hist;
  int64_t done = 0;
  double nh = NAN, nc = NAN;
  int conv = 0;
  while (done < max_steps && !conv) {
    int rc = mclbm_step(h, check_every);
    if (rc != MCLBM_OK) return rc;
    done += check_every;
    if ((rc = mclbm_nusselt(h, &nh, &nc)) != MCLBM_OK) return rc;
    hist.push_back(nh);
    conv = steady(hist.data(), (int64_t)hist.size(), tol, lags, n_lags);
  }
  if (steps) *steps = done;
  if (nu_hot) *nu_hot = nh;
  if (nu_cold) *nu_cold = nc;
  if (converged) *converged = conv;
  return MCLBM_OK;
}

int mclbm_batch_run_to_steady(mclbm_batch_t* b, double tol, int64_t check_every,
                              int64_t max_steps, const int32_t* lags, int n_lags, int64_t* steps,
                              double* nu_hot, int64_t* total_steps) {
  if (!lags) {
    lags = kDefaultLags;
    n_lags = 2;
  }
  if (!b || check_every < 2 || check_every % 2 || max_steps < 0 || !args_ok(tol, lags, n_lags))
    return MCLBM_EINVAL;
  const int n = mcl::batch_size(b);
  if (n < 1) return MCLBM_EINVAL;
  std::vector<std::vector<double>> hist(n);
  std::vector<int> active(n, 1);
  std::vector<int64_t> at(n, -1);
  std::vector<double> hot(n), cold(n), last(n, NAN);
  int64_t done = 0;
  int left = n;
  while (left > 0 && done < max_steps) {
    int rc = mclbm_batch_step(b, check_every);
    if (rc != MCLBM_OK) return rc;
    done += check_every;
    if ((rc = mclbm_batch_nusselt(b, hot.data(), cold.data())) != MCLBM_OK) return rc;
    bool changed = false;
    for (int c = 0; c < n; ++c) {
      if (!active[c]) continue;
      hist[c].push_back(hot[c]);
      last[c] = hot[c];
      if (steady(hist[c].data(), (int64_t)hist[c].size(), tol, lags, n_lags)) {
        active[c] = 0;
        at[c] = done;
        --left;
        changed = true;
      }
    }
    if (changed && left > 0 && (rc = mclbm_batch_set_active(b, active.data())) != MCLBM_OK)
      return rc;
  }
  for (int c = 0; c < n; ++c) {
    if (steps) steps[c] = at[c];
    if (nu_hot) nu_hot[c] = last[c];
  }
  if (total_steps) *total_steps = done;
  return MCLBM_OK;
}

}  // extern "C"
