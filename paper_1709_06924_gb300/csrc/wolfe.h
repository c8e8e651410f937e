// wolfe.h -- the strong-Wolfe line search of More & Thuente (1994), as a
// resumable state machine (host code).
//
// On the auxiliary function psi(a) = phi(a) - phi(0) - ftol a phi'(0) until
// a step with psi <= 0 and phi' >= 0 (up to ftol/gtol) is seen, then on phi;
// the interval of uncertainty is updated with safeguarded cubic / quadratic
// / secant steps and bisected when it fails to shrink by 2/3.  A trial point
// that is not a valid tessellation counts as a failed evaluation: the step is
// halved toward the best point so far and never exceeded again.
//
// Use: r = begin(f0, d0, a0); while (r == 0) { evaluate phi at trial();
// r = feed(cb, f, d); }.  cb = 0 valid (f, d given), 1 invalid trial point,
// < 0 hard failure.  Result: 1 strong Wolfe, 2 width below xtol, 3 maxfev,
// 4 at amin, 5 at amax, 6 rounding, 7 bad input, -1 callback failure; the
// last evaluated point is (last_a, last_f, last_d) with last_f = +inf if it
// was invalid.  Many searches can be stepped in lockstep, one per problem.
#pragma once

#include <math.h>

#include <algorithm>

namespace scvt {

class WolfeSearch {
  public:
    double ftol = 1e-4, gtol = 0.9, xtol = 1e-16, amin = 1e-20, amax = 1e20;
    int maxfev = 10;
    double last_a = 0.0, last_f = 0.0, last_d = 0.0;
    int nfev = 0;

    int begin(double f0, double d0, double a0) {
        nfev = 0;
        last_a = a0;
        last_f = f0;
        last_d = d0;
        if (!(d0 < 0.0) || !(a0 > 0.0)) return 7;
        f0_ = f0;
        d0_ = d0;
        lo_ = {0.0, f0, d0};
        hi_ = {0.0, f0, d0};
        brack_ = false;
        first_stage_ = true;
        slope_ = ftol * d0;
        width_ = amax - amin;
        width_prev_ = 2.0 * width_;
        lo_bound_ = 0.0;
        hi_bound_ = a0 * 5.0;
        cap_ = INFINITY;
        a_ = a0;
        prepare();
        return 0;
    }

    double trial() const { return a_; }

    int feed(int cb, double f, double d) {
        ++nfev;
        last_a = a_;
        last_f = f;
        last_d = d;
        if (cb < 0) return -1;
        if (cb > 0) {
            last_f = INFINITY;
            if (nfev >= maxfev) return 3;
            cap_ = a_;
            a_ = lo_.a + 0.5 * (a_ - lo_.a);
            prepare();
            return 0;
        }
        const double a = a_;
        const double armijo = f0_ + a * slope_;
        int info = 0;
        if (brack_ && (a <= lo_bound_ || a >= hi_bound_)) info = 6;
        if (a == amax && f <= armijo && d <= slope_) info = 5;
        if (a == amin && (f > armijo || d >= slope_)) info = 4;
        if (nfev >= maxfev) info = 3;
        if (brack_ && hi_bound_ - lo_bound_ <= xtol * hi_bound_) info = 2;
        if (f <= armijo && fabs(d) <= gtol * (-d0_)) info = 1;
        if (info) return info;
        if (first_stage_ && f <= armijo && d >= std::min(ftol, gtol) * d0_) first_stage_ = false;
        double next;
        if (first_stage_ && f <= lo_.f && f > armijo) {
            // work on psi: shift values and slopes by the Armijo line
            Pt l = {lo_.a, lo_.f - lo_.a * slope_, lo_.d - slope_};
            Pt u = {hi_.a, hi_.f - hi_.a * slope_, hi_.d - slope_};
            Pt t = {a, f - a * slope_, d - slope_};
            std::swap(l, lo_);
            std::swap(u, hi_);
            next = update(t);
            lo_ = {lo_.a, lo_.f + lo_.a * slope_, lo_.d + slope_};
            hi_ = {hi_.a, hi_.f + hi_.a * slope_, hi_.d + slope_};
        } else {
            next = update({a, f, d});
        }
        if (brack_) {
            if (fabs(hi_.a - lo_.a) >= 0.66 * width_prev_) next = lo_.a + 0.5 * (hi_.a - lo_.a);
            width_prev_ = width_;
            width_ = fabs(hi_.a - lo_.a);
            lo_bound_ = std::min(lo_.a, hi_.a);
            hi_bound_ = std::max(lo_.a, hi_.a);
        } else {
            lo_bound_ = lo_.a;
            hi_bound_ = next + 4.0 * (next - lo_.a);
        }
        a_ = next;
        prepare();
        return 0;
    }

    // run to completion with a synchronous evaluator phi(a, f, d) -> cb
    template <class Phi>
    int run(Phi &&phi, double f0, double d0, double &a, double &f, double &d, int &nf) {
        int r = begin(f0, d0, a);
        while (r == 0) {
            double ft = 0.0, dt = 0.0;
            const int cb = phi(a_, ft, dt);
            r = feed(cb, ft, dt);
        }
        a = last_a;
        f = last_f;
        d = last_d;
        nf = nfev;
        return r;
    }

  private:
    struct Pt {
        double a, f, d;
    };
    Pt lo_{}, hi_{};  // best point so far and the other end of the interval
    bool brack_ = false, first_stage_ = true;
    double f0_ = 0.0, d0_ = 0.0, slope_ = 0.0, width_ = 0.0, width_prev_ = 0.0;
    double lo_bound_ = 0.0, hi_bound_ = 0.0, cap_ = INFINITY, a_ = 0.0;

    // the step to evaluate next: clamped, below the smallest invalid step,
    // and the best point itself when the interval is exhausted
    void prepare() {
        a_ = std::min(std::max(a_, amin), amax);
        if (a_ >= cap_) a_ = lo_.a + 0.5 * (cap_ - lo_.a);
        const bool last_chance = nfev >= maxfev - 1;
        if ((brack_ && (a_ <= lo_bound_ || a_ >= hi_bound_)) || last_chance ||
            (brack_ && hi_bound_ - lo_bound_ <= xtol * hi_bound_))
            a_ = lo_.a;
    }

    // minimiser of the cubic through (x, fx, dx) and (t, ft, dt), in the
    // theta / gamma form; ok = false when it does not exist
    static double cubic(const Pt &x, const Pt &t, bool &ok) {
        double theta = 3.0 * (x.f - t.f) / (t.a - x.a) + x.d + t.d;
        double sc = std::max(fabs(theta), std::max(fabs(x.d), fabs(t.d)));
        double rad = (theta / sc) * (theta / sc) - (x.d / sc) * (t.d / sc);
        ok = rad > 0.0;
        double gamma = sc * sqrt(std::max(rad, 0.0));
        if (t.a < x.a) gamma = -gamma;
        double p = (gamma - x.d) + theta;
        double q = ((gamma - x.d) + gamma) + t.d;
        if (q == 0.0) {
            ok = false;
            return x.a;
        }
        return x.a + (p / q) * (t.a - x.a);
    }

    double update(Pt t) {
        const Pt &x = lo_;
        const double sx = (x.d > 0.0) - (x.d < 0.0);
        const bool opposite = t.d * sx < 0.0;
        bool ok;
        double nxt;
        if (t.f > x.f) {
            double ac = cubic(x, t, ok);
            double aq = x.a + (x.d / ((x.f - t.f) / (t.a - x.a) + x.d)) / 2.0 * (t.a - x.a);
            nxt = (fabs(ac - x.a) < fabs(aq - x.a)) ? ac : ac + (aq - ac) / 2.0;
            brack_ = true;
        } else if (opposite) {
            double ac = cubic(x, t, ok);
            double as = t.a + t.d / (t.d - x.d) * (x.a - t.a);
            nxt = (fabs(ac - t.a) > fabs(as - t.a)) ? ac : as;
            brack_ = true;
        } else if (fabs(t.d) < fabs(x.d)) {
            double ac = cubic(x, t, ok);
            bool beyond = ok && ((t.a > x.a) ? (ac > t.a) : (ac < t.a));
            if (!beyond) ac = (t.a > x.a) ? hi_bound_ : lo_bound_;
            double as = t.a + t.d / (t.d - x.d) * (x.a - t.a);
            if (brack_) {
                nxt = (fabs(ac - t.a) < fabs(as - t.a)) ? ac : as;
                nxt = (t.a > x.a) ? std::min(t.a + 0.66 * (hi_.a - t.a), nxt)
                                  : std::max(t.a + 0.66 * (hi_.a - t.a), nxt);
            } else {
                nxt = (fabs(ac - t.a) > fabs(as - t.a)) ? ac : as;
                nxt = std::min(hi_bound_, std::max(lo_bound_, nxt));
            }
        } else {
            if (brack_) nxt = cubic(t, hi_, ok);
            else nxt = (t.a > x.a) ? hi_bound_ : lo_bound_;
        }
        if (t.f > x.f) {
            hi_ = t;
        } else {
            if (opposite) hi_ = lo_;
            lo_ = t;
        }
        return nxt;
    }
};

}  // namespace scvt
