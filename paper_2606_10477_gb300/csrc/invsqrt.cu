// CryptoInvSqrt (Alg. 1) with the pre-normalisation of Sec. 2.3:
//   t   = affine map of a/B onto [-1, 1]            (one level)
//   x   = 0.5 * a / B                                (ct_x, one level)
//   y0  = sum_j c_j T_j(t), c_j the Chebyshev interpolant of 1/sqrt on [lo/B, hi/B]
//   y  <- 1.5 y - x y^3   (Newton, Sec. 2.2; two levels per step)
//   out = y / sqrt(B)
//
// The Chebyshev sum is evaluated in the Chebyshev basis with baby steps
// T_1..T_k (k = 2^ceil(m/2), m = ceil(log2(d+1))) and giant steps T_k, T_2k, ...
// (Paterson-Stockmeyer in the form of Bossuat et al. 2021): a polynomial of
// degree D >= G is split as p = q T_G + r with
//   q_0 = c_G, q_i = 2 c_{G+i},  r_i = c_i - c_{2G-i} (when 2G-i <= D),
// from 2 T_G T_{j-G} = T_j + T_{2G-j}.  Each partial result is produced at a
// prescribed (level, scale) so that additions never need a correction.  Two
// plans: fewest products (every polynomial below the baby-step degree is a leaf,
// its constant products of T_1..T_D summed at one level below the lowest T_j:
// ceil(log2(d+1)) + 1 levels for most d) and fewest levels (such a polynomial is
// a leaf only when that reaches the level asked of it, else it is split again at
// the largest power of two <= D, so that the constants multiply lower T_j's with
// a level to spare: ceil(log2(d+1)) levels, i.e. degree 2^{d_e} - 2 in d_e
// levels as the paper's libraries, Sec. 4.3, for a few more products).  The
// fewest-products plan is taken when it ends at a level >= `need`.
#include <cmath>

#include "internal.cuh"

namespace hedap {

typedef std::unique_ptr<Ct> CtP;

// Chebyshev interpolation coefficients of 1/sqrt(x) at the d+1 first-kind nodes on [lo, hi]
static std::vector<double> cheb_interp(double lo, double hi, int d) {
  const int n = d + 1;
  std::vector<double> f(n), c(n);
  for (int k = 0; k < n; ++k) {
    const double node = 0.5 * (lo + hi) + 0.5 * (hi - lo) * std::cos(M_PI * (k + 0.5) / n);
    f[k] = 1.0 / std::sqrt(node);
  }
  for (int j = 0; j < n; ++j) {
    double acc = 0;
    for (int k = 0; k < n; ++k) acc += f[k] * std::cos(M_PI * j * (k + 0.5) / n);
    c[j] = (j == 0 ? 1.0 : 2.0) / n * acc;
  }
  return c;
}

struct ChebPS {
  Ctx& C;
  std::map<int, CtP> T;
  std::vector<int> giants;
  int k = 2;
  explicit ChebPS(Ctx& c) : C(c) {}

  static int degree(const std::vector<double>& p) { return (int)p.size() - 1; }
  int giant(int D) const {
    int g = 0;
    for (int v : giants)
      if (v <= D) g = v;
    return g;
  }
  // the split point of a degree-D polynomial: the largest giant step <= D, or, below the baby-step
  // degree, the largest power of two <= D
  int split_at(int D) const {
    if (D >= k) return giant(D);
    int g = 1;
    while (2 * g <= D) g *= 2;
    return g;
  }
  static void divide(const std::vector<double>& p, int G, std::vector<double>& qt, std::vector<double>& rm) {
    const int D = degree(p);
    qt.assign(D - G + 1, 0.0);
    qt[0] = p[G];
    for (int i = 1; i <= D - G; ++i) qt[i] = 2.0 * p[G + i];
    rm.assign(p.begin(), p.begin() + G);
    for (int i = 0; i < G; ++i)
      if (2 * G - i <= D) rm[i] -= p[2 * G - i];
  }
  // level of a leaf sum over T_1 .. T_D: one below the lowest of them
  int leaf_level(int D) const {
    int lv = INT_MAX;
    for (int j = 1; j <= D; ++j) lv = std::min(lv, T.at(j)->level - 1);
    return lv;
  }
  bool fewest_levels = false;  // the plan (see above)
  bool leaf_at(int D, int level) const { return D < k && (!fewest_levels || D < 2 || leaf_level(D) >= level); }
  // highest level p can be produced at: below the baby-step degree a leaf or (fewest levels) the better
  // of a leaf and a split
  int top_level(const std::vector<double>& p) const {
    const int D = degree(p);
    const int leaf = D < k ? leaf_level(D) : INT_MIN;
    if (D < k && (!fewest_levels || D < 2)) return leaf;
    const int G = split_at(D);
    std::vector<double> qt, rm;
    divide(p, G, qt, rm);
    const int lq = degree(qt) == 0 ? INT_MAX : top_level(qt);
    return std::max(leaf, std::min(std::min(lq, T.at(G)->level) - 1, top_level(rm)));
  }
  // p at (level + 1, label scale * q_{level+1}) before its final rescale: the leaf sums c_j T_j as
  // unrescaled products plus c_0, an inner node adds the relinearised q T_G to the unrescaled r,
  // so a whole evaluation ends with one rescale per product of the recursion and one more
  CtP eval_raw(const std::vector<double>& p, int level, double scale) {
    const int D = degree(p);
    const double raw = scale * (double)C.primes[level + 1];
    if (leaf_at(D, level)) {  // one pass over T_1 .. T_D (read at level + 1 in place)
      std::vector<std::pair<const Ct*, double>> terms;
      for (int j = 1; j <= D; ++j) terms.emplace_back(T.at(j).get(), p[j]);
      return ev_lincomb_raw(C, terms, level + 1, scale, p[0]);
    }
    const int G = split_at(D);
    std::vector<double> qt, rm;
    divide(p, G, qt, rm);
    const Ct& tg = *T.at(G);
    CtP prod;
    if (degree(qt) == 0) {
      prod = ev_lincomb_raw(C, {{&tg, qt[0]}}, level + 1, scale, 0.0);
    } else {
      const double sq = scale * (double)C.primes[level + 1] / tg.scale;
      CtP qv = eval(qt, level + 1, sq);
      prod = ev_mul_relin(C, *qv, tg);  // at min level = level + 1
    }
    prod->scale = raw;
    CtP rv = eval_raw(rm, level, scale);
    return ev_add(C, *prod, *rv, false);
  }
  CtP eval(const std::vector<double>& p, int level, double scale) {
    CtP r;
    const int D = degree(p);
    if (!leaf_at(D, level)) {  // an inner node: its product's ModDown is fused into this rescale
      const int G = split_at(D);
      std::vector<double> qt, rm;
      divide(p, G, qt, rm);
      if (degree(qt) > 0) {
        const Ct& tg = *T.at(G);
        const double raw = scale * (double)C.primes[level + 1];
        CtP qv = eval(qt, level + 1, raw / tg.scale);
        CtP rv = eval_raw(rm, level, scale);
        const int lp = std::min(qv->level, tg.level);
        if (rv->level == lp) {
          // prod + rv with both constants round(out q / raw) = 1, out = raw / q_lp
          r = ev_mul_lincomb_rescale(C, *qv, tg, raw, 1.0, {{rv.get(), 1.0}}, raw / (double)C.primes[lp], 0.0);
        } else {
          CtP prod = ev_mul_relin(C, *qv, tg);
          prod->scale = raw;
          r = ev_rescale(C, *ev_add(C, *prod, *rv, false));
        }
      }
    }
    if (!r) r = ev_rescale(C, *eval_raw(p, level, scale));
    r->scale = scale;
    return r;
  }
  // 2 T_a T_b - T_c, with T_c the constant 1 when c == 0; for c > 0 the product and 0.5 T_c are
  // subtracted before the rescale (one rescale for both)
  CtP product(const Ct& ta, const Ct& tb, int c) {
    CtP diff;
    if (c == 0) {
      return ev_add_const_mul_int(C, *ev_mul(C, ta, tb), -0.5, 2);
    } else {
      const int l = std::min(ta.level, tb.level);
      const double ps = ta.scale * tb.scale, out = ps / (double)C.primes[l];
      // pr * 1 - 0.5 T_c in one pass (the constant of pr is round(sp) = 1, sp = out q_l / pr.scale),
      // the product's ModDown fused into the rescale
      diff = ev_mul_lincomb_rescale(C, ta, tb, ps, 1.0, {{T.at(c).get(), -0.5}}, out, 0.0);
      diff->scale = out;
    }
    return ev_mul_int(C, *diff, 2);
  }
  CtP run(const Ct& t, const std::vector<double>& coeffs, double target, int need) {
    const int d = degree(coeffs);
    int m = 0;
    while ((1 << m) < d + 1) ++m;
    const int lb = std::max(1, (m + 1) / 2);
    k = 1 << lb;
    T.clear();
    T[1] = ct_copy(C, t, t.level);
    for (int j = 2; j <= k; ++j) T[j] = (j % 2 == 0) ? product(*T.at(j / 2), *T.at(j / 2), 0)
                                                     : product(*T.at(j / 2), *T.at(j / 2 + 1), 1);
    giants.clear();
    for (int g = k; g < (1 << m); g *= 2) {
      giants.push_back(g);
      if (!T.count(g)) T[g] = product(*T.at(g / 2), *T.at(g / 2), 0);
    }
    fewest_levels = need < 0;
    int lvl = top_level(coeffs);
    if (!fewest_levels && lvl < need) {
      fewest_levels = true;
      lvl = top_level(coeffs);
    }
    if (lvl < 0) throw Error(HEDAP_ERR_LEVEL, "Chebyshev evaluation: not enough levels");
    return eval(coeffs, lvl, target);
  }
};

std::unique_ptr<Ct> cheb_eval(Ctx& C, const Ct& t, const std::vector<double>& coeffs, double target, int need) {
  ChebPS ps(C);
  return ps.run(t, coeffs, target, need);
}

// One Newton step in Alg. 1's loop order; tmp_alpha = 1.5 y is produced last, at the level of
// the relinearised tmp_beta and labelled with its scale, and tmp_alpha - tmp_beta is rescaled once.
static CtP newton_step(Ctx& C, const Ct& x, const Ct& y) {
  CtP yy = ev_mul(C, y, y);
  CtP xy = ev_mul(C, x, y);
  const int l = std::min(xy->level, yy->level);
  const double ps = xy->scale * yy->scale, out = ps / (double)C.primes[l];
  // 1.5 y - tmp_beta in one pass (the constant of tmp_beta is -round(sp) = -1, sp = out q_l / tb.scale),
  // tmp_beta's ModDown fused into the rescale
  CtP r = ev_mul_lincomb_rescale(C, *xy, *yy, ps, -1.0, {{&y, 1.5}}, out, 0.0);
  r->scale = out;
  return r;
}

// Bootstrapping placement (the Pre-BTS indicator c of Sec. 4.1 and BTS during
// the Newton loop, Sec. 4.3): pre_bts bootstraps a/B first; bit j (< 62) of
// bts_mask bootstraps y before Newton step j (bit 0: right after the Chebyshev
// step, as in Alg. 1); bit 63 bootstraps lazily, before any step that would
// leave y below level 1 (y has fewer than 3 levels), so that a later bootstrap
// stays possible and the state after i steps does not depend on how many steps
// follow.  ct_x is not bootstrapped in Alg. 1 (a Newton output sits two levels
// below it); bit 62 (a variant) bootstraps it too whenever y is bootstrapped and
// x has fewer than 5 levels, scaled by the power of two bounding x = 0.5 a/B.
// Y, the power of two bounding y, scales
// y into [-1, 1] around each BTS.  The final 1/sqrt(B) is applied to the scale
// label (no level is used).
InvSqrtRun::InvSqrtRun(Ctx& C_, const Ct& in, const hedap_invsqrt_cfg& c) : C(C_), cfg(c) {
  if (!(cfg.B > 0) || !(cfg.lo > 0) || !(cfg.hi > cfg.lo) || cfg.degree < 1 || cfg.degree > 4096 ||
      ((size_t)1 << std::min(cfg.log_slots, 40u)) > C.N / 2)
    throw Error(HEDAP_ERR_ARG, "invsqrt: invalid configuration");
  if ((cfg.pre_bts || cfg.bts_mask) && !C.bts)
    throw Error(HEDAP_ERR_ARG, "invsqrt: bootstrapping not configured on this context");
  lo = cfg.lo / cfg.B;
  hi = cfg.hi / cfg.B;
  Y = 1;
  while ((double)Y < 1.0 / std::sqrt(lo)) Y *= 2;
  double Bf = cfg.B;
  CtP pre;
  if (cfg.pre_bts) {  // a -> BTS(a / B), values in (0, 1]
    if (in.level < 1) throw Error(HEDAP_ERR_LEVEL, "invsqrt: input level too low");
    CtP d = in.level > 1 ? ev_drop(C, in, 1) : nullptr;
    pre = bootstrap_core(C, *ev_mul_const(C, d ? *d : in, 1.0 / cfg.B, (double)C.primes[0] / 4096.0),
                         (int)cfg.log_slots);
    Bf = 1.0;
  }
  const Ct& a = pre ? *pre : in;
  if (a.level < 2) throw Error(HEDAP_ERR_LEVEL, "invsqrt: input level too low");
  const double alpha = 2.0 / (Bf * (hi - lo)), beta = -(hi + lo) / (hi - lo);
  t = ev_add_const(C, *ev_mul_const(C, a, alpha, C.scale), beta);
  x = ev_mul_const(C, a, 0.5 / Bf, C.scale);
}
// with bootstrapping in the configuration, the fewest-levels plan (a level saved is a bootstrap saved or
// postponed); without, the fewest products while the Newton steps still fit (two levels each)
void InvSqrtRun::chebyshev() {
  const int need = (cfg.pre_bts || cfg.bts_mask) ? -1 : 2 * (int)cfg.newton_iters;
  y = cheb_eval(C, *t, cheb_interp(lo, hi, (int)cfg.degree), C.scale, need);
}
void InvSqrtRun::newton(int i) {
  const bool force = i < 62 && ((cfg.bts_mask >> i) & 1);
  const bool lazy = ((cfg.bts_mask >> 63) & 1) && y->level < 3;
  if (force || lazy) {
    y = bootstrap_scaled(C, *y, Y, (int)cfg.log_slots);
    if (((cfg.bts_mask >> 62) & 1) && x->level < 5) {  // variant: ct_x refreshed with y
      i64 Yx = 1;
      while ((double)Yx < 0.5 * hi) Yx *= 2;
      x = bootstrap_scaled(C, *x, Yx, (int)cfg.log_slots);
    }
  }
  if (std::min(y->level, x->level) < 2) throw Error(HEDAP_ERR_LEVEL, "invsqrt: level exhausted in Newton loop");
  y = newton_step(C, *x, *y);
}
std::unique_ptr<Ct> InvSqrtRun::result() const {
  auto r = ct_copy(C, *y, y->level);
  if (cfg.B != 1.0) r->scale *= std::sqrt(cfg.B);
  return r;
}

std::unique_ptr<Ct> invsqrt(Ctx& C, const Ct& in, const hedap_invsqrt_cfg& cfg) {
  InvSqrtRun run(C, in, cfg);
  run.chebyshev();
  const int n = (int)cfg.newton_iters;
  for (int i = 0; i < n; ++i) run.newton(i);
  if (n == 0 && (cfg.bts_mask & 1)) run.y = bootstrap_scaled(C, *run.y, run.Y, (int)cfg.log_slots);
  if (cfg.B != 1.0) run.y->scale *= std::sqrt(cfg.B);
  return std::move(run.y);
}

// CryptoInvSqrt of many single ciphertexts, each at its own level (no level is dropped).  Members with
// equal input level, scale and configuration form a batch (input order, up to 16); after every stage --
// the pre-normalisation with its Pre-BTS, the Chebyshev step, each Newton step -- batches of one
// configuration whose carried ciphertexts (x, y, and t before the Chebyshev step) stand at equal
// levels and scales are merged into one (up to 16 members).  Members whose inputs differ in level
// meet where the algorithm brings them to the same level: after a Pre-BTS (all at the bootstrapped
// level), or never when the configuration keeps ct_x at its input level (Alg. 1).  Every member's
// result equals its own invsqrt() bit for bit: batches and merges only pack identical computations.
std::vector<std::unique_ptr<Ct>> invsqrt_mixed(Ctx& C, const std::vector<const Ct*>& in,
                                               const std::vector<hedap_invsqrt_cfg>& cfgs) {
  struct Batch {
    std::vector<size_t> m;  // members, in batch order
    std::unique_ptr<InvSqrtRun> r;
  };
  const size_t n = in.size();
  if (cfgs.size() != n) throw Error(HEDAP_ERR_ARG, "one configuration per input");
  for (const Ct* c : in)
    if (!c || c->batch != 1) throw Error(HEDAP_ERR_ARG, "inputs must be single ciphertexts");
  std::vector<Batch> bs;
  std::vector<bool> taken(n, false);
  for (size_t i = 0; i < n; ++i) {
    if (taken[i]) continue;
    Batch b;
    for (size_t j = i; j < n && b.m.size() < (size_t)kMaxBatchCts; ++j)
      if (!taken[j] && in[j]->level == in[i]->level && in[j]->scale == in[i]->scale && same_cfg(cfgs[i], cfgs[j])) {
        b.m.push_back(j);
        taken[j] = true;
      }
    std::unique_ptr<Ct> packed;
    if (b.m.size() > 1) {
      std::vector<const Ct*> v;
      for (size_t j : b.m) v.push_back(in[j]);
      packed = batch_pack(C, v);
    }
    b.r.reset(new InvSqrtRun(C, packed ? *packed : *in[i], cfgs[i]));
    bs.push_back(std::move(b));
  }
  auto same_state = [](const std::unique_ptr<Ct>& a, const std::unique_ptr<Ct>& b) {
    return (!a && !b) || (a && b && a->level == b->level && a->scale == b->scale);
  };
  auto merge = [&]() {
    for (size_t a = 0; a < bs.size(); ++a)
      for (size_t b = a + 1; b < bs.size();) {
        InvSqrtRun &ra = *bs[a].r, &rb = *bs[b].r;
        if (!same_cfg(cfgs[bs[a].m[0]], cfgs[bs[b].m[0]]) || !same_state(ra.t, rb.t) || !same_state(ra.x, rb.x) ||
            !same_state(ra.y, rb.y) || bs[a].m.size() + bs[b].m.size() > (size_t)kMaxBatchCts) {
          ++b;
          continue;
        }
        for (std::unique_ptr<Ct>* f : {&ra.t, &ra.x, &ra.y}) {
          std::unique_ptr<Ct>& g = f == &ra.t ? rb.t : f == &ra.x ? rb.x : rb.y;
          if (*f) *f = batch_pack(C, {f->get(), g.get()});
        }
        bs[a].m.insert(bs[a].m.end(), bs[b].m.begin(), bs[b].m.end());
        bs.erase(bs.begin() + (long)b);
      }
  };
  merge();
  for (Batch& b : bs) {
    b.r->chebyshev();
    b.r->t.reset();  // needed by the Chebyshev step only
  }
  merge();
  for (int i = 0;; ++i) {
    bool any = false;
    for (Batch& b : bs)
      if (i < (int)b.r->cfg.newton_iters) {
        b.r->newton(i);
        any = true;
      }
    if (!any) break;
    merge();
  }
  std::vector<std::unique_ptr<Ct>> out(n);
  for (Batch& b : bs) {
    InvSqrtRun& r = *b.r;
    if (r.cfg.newton_iters == 0 && (r.cfg.bts_mask & 1)) r.y = bootstrap_scaled(C, *r.y, r.Y, (int)r.cfg.log_slots);
    if (r.cfg.B != 1.0) r.y->scale *= std::sqrt(r.cfg.B);
    for (size_t k = 0; k < b.m.size(); ++k)
      out[b.m[k]] = b.m.size() > 1 ? batch_unpack(C, *r.y, (int)k) : std::move(r.y);
  }
  return out;
}

}  // namespace hedap
