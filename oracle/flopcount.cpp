/*
 * Counting build of the oracle (test and measurement infrastructure, like the
 * oracle itself): mgrit_oracle.c compiled unchanged as C++ with `double`
 * replaced by a number type that counts the floating-point operations the
 * oracle performs on data.  This gives the algorithmic work of one time step
 * Phi (Sec. 2.2, Eq. SSPRK3, through Eq. spaceDisc, the WENO5 tables of
 * Sec. 2.1.1 and the Lax-Friedrichs flux of Sec. 2.1.2) as the paper's
 * formulas state it, the per-unit figure of the roofline of the relaxation
 * kernel.
 *
 * Counting rules (those of a compiler that folds constants):
 *  - a value is either data (derived from the input state) or a constant
 *    (literals, the printed tables, dt, dx and anything computed from them
 *    alone); operations on constants only are folded and not counted;
 *  - x * 0 is the constant 0, x * 1 and x * (-1) are x and -x, x + 0, x - 0
 *    and x / 1 are x: not counted (the oracle's smoothness-indicator quadratic
 *    forms act on the stencil minus its middle value, whose middle entry is
 *    the literal 0);
 *  - every other +, -, *, / with a data operand counts 1, as do |x|, sqrt and
 *    each comparison of data (the maxima of the Lax-Friedrichs speed);
 *    negation is free.
 * Build and run: python oracle/count_flops.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cstdio>

namespace fcount {
enum { ADD, MUL, DIV, ABS, CMP, SQRT, NKIND };
static long long g_n[NKIND];
}  // namespace fcount

struct fc {
    double v;
    bool k;   // constant (not derived from data)
    fc() : v(0.0), k(true) {}
    fc(double x) : v(x), k(true) {}
    static fc data(double x)
    {
        fc r(x);
        r.k = false;
        return r;
    }
};

static inline fc mk(double v, bool k)
{
    fc r(v);
    r.k = k;
    return r;
}
static inline bool is_c(const fc &a, double c) { return a.k && a.v == c; }

static inline fc operator+(fc a, fc b)
{
    if (a.k && b.k) return mk(a.v + b.v, true);
    if (is_c(a, 0.0)) return b;
    if (is_c(b, 0.0)) return a;
    ++fcount::g_n[fcount::ADD];
    return mk(a.v + b.v, false);
}
static inline fc operator-(fc a) { return mk(-a.v, a.k); }
static inline fc operator-(fc a, fc b)
{
    if (a.k && b.k) return mk(a.v - b.v, true);
    if (is_c(b, 0.0)) return a;
    if (is_c(a, 0.0)) return -b;
    ++fcount::g_n[fcount::ADD];
    return mk(a.v - b.v, false);
}
static inline fc operator*(fc a, fc b)
{
    if (a.k && b.k) return mk(a.v * b.v, true);
    if (is_c(a, 0.0) || is_c(b, 0.0)) return mk(a.v * b.v, true);
    if (is_c(a, 1.0)) return b;
    if (is_c(b, 1.0)) return a;
    if (is_c(a, -1.0)) return -b;
    if (is_c(b, -1.0)) return -a;
    ++fcount::g_n[fcount::MUL];
    return mk(a.v * b.v, false);
}
static inline fc operator/(fc a, fc b)
{
    if (a.k && b.k) return mk(a.v / b.v, true);
    if (is_c(b, 1.0)) return a;
    ++fcount::g_n[fcount::DIV];
    return mk(a.v / b.v, false);
}
static inline fc &operator+=(fc &a, fc b) { return a = a + b; }
static inline fc &operator-=(fc &a, fc b) { return a = a - b; }
static inline fc &operator*=(fc &a, fc b) { return a = a * b; }
static inline fc &operator/=(fc &a, fc b) { return a = a / b; }

static inline bool cmp_count(const fc &a, const fc &b)
{
    if (!(a.k && b.k)) ++fcount::g_n[fcount::CMP];
    return true;
}
static inline bool operator<(fc a, fc b) { return cmp_count(a, b) && a.v < b.v; }
static inline bool operator>(fc a, fc b) { return cmp_count(a, b) && a.v > b.v; }
static inline bool operator<=(fc a, fc b) { return cmp_count(a, b) && a.v <= b.v; }
static inline bool operator>=(fc a, fc b) { return cmp_count(a, b) && a.v >= b.v; }
static inline bool operator==(fc a, fc b) { return cmp_count(a, b) && a.v == b.v; }
static inline bool operator!=(fc a, fc b) { return cmp_count(a, b) && a.v != b.v; }

static inline fc fabs(fc a)
{
    if (a.k) return mk(fabs(a.v), true);
    ++fcount::g_n[fcount::ABS];
    return mk(fabs(a.v), false);
}
static inline fc sqrt(fc a)
{
    if (a.k) return mk(sqrt(a.v), true);
    ++fcount::g_n[fcount::SQRT];
    return mk(sqrt(a.v), false);
}
static inline bool isfinite(fc a) { return isfinite(a.v); }

#define double fc
#include "mgrit_oracle.c"
#undef double

// Operations of one oracle step orc_step (scheme, flux, numflux as in the
// oracle) on the nx-cell state u; counts[0..5] = additions/subtractions,
// multiplications, divisions, |x|, comparisons, square roots; out (nx
// values) receives the step's result, the oracle's own arithmetic.
extern "C" void fc_count_step(int nx, double Lx, double dt, int scheme, int flux, int numflux,
                              const double *u, long long *counts, double *res)
{
    fc *in = new fc[nx], *out = new fc[nx];
    for (int i = 0; i < nx; ++i) in[i] = fc::data(u[i]);
    for (int k = 0; k < fcount::NKIND; ++k) fcount::g_n[k] = 0;
    orc_step(nx, fc(Lx), fc(dt), scheme, flux, numflux, in, out);
    for (int k = 0; k < fcount::NKIND; ++k) counts[k] = fcount::g_n[k];
    for (int i = 0; i < nx; ++i) res[i] = out[i].v;
    delete[] in;
    delete[] out;
}

// The same for one transposed step orc_step_vjp (split numerical flux).
extern "C" void fc_count_step_vjp(int nx, double Lx, double dt, int scheme, int flux,
                                  const double *u, const double *lam, long long *counts)
{
    fc *in = new fc[nx], *l = new fc[nx], *out = new fc[nx];
    for (int i = 0; i < nx; ++i) {
        in[i] = fc::data(u[i]);
        l[i] = fc::data(lam[i]);
    }
    for (int k = 0; k < fcount::NKIND; ++k) fcount::g_n[k] = 0;
    orc_step_vjp(nx, fc(Lx), fc(dt), scheme, flux, in, l, out);
    for (int k = 0; k < fcount::NKIND; ++k) counts[k] = fcount::g_n[k];
    delete[] in;
    delete[] l;
    delete[] out;
}
