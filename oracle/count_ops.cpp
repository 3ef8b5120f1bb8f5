/*
 * count_ops.cpp -- the oracle with every floating-point operation counted.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle itself.  This file compiles
 * wb_oracle.c unchanged as C++ with `double` standing for `cdouble`, a value
 * type that behaves as an IEEE double and counts the operations applied to
 * it.  The result is the algorithmic operation count of the oracle's own
 * steps (Sec. 2.1, 2.2), per interface or per zone update, with
 *   add/sub, mul  counted one each unless an operand is exactly 0 or +-1
 *                 (the structural zeros and signs of the dense eigenvector
 *                 matrices and of dU/dW do no work);
 *   div, sqrt     counted separately;
 *   negation, |x|, comparisons, min/max  not counted.
 * The oracle has no fused multiply-adds (it is built with -ffp-contract=off);
 * an FMA elsewhere counts as one mul and one add here.
 * Counters are plain globals: call the counted functions from one thread.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

namespace {
long long n_add = 0, n_mul = 0, n_div = 0, n_sqrt = 0;

inline bool trivial_add(double a) { return a == 0.0; }
inline bool trivial_mul(double a) { return a == 0.0 || a == 1.0 || a == -1.0; }
}  // namespace

struct cdouble {
    double v;
    cdouble() = default;
    constexpr cdouble(double x) : v(x) {}
    explicit constexpr operator long() const { return (long)v; }
    explicit constexpr operator int() const { return (int)v; }
    cdouble& operator+=(cdouble b);
    cdouble& operator-=(cdouble b);
    cdouble& operator*=(cdouble b);
    cdouble& operator/=(cdouble b);
};

inline cdouble operator+(cdouble a, cdouble b) {
    if (!trivial_add(a.v) && !trivial_add(b.v)) n_add++;
    return cdouble(a.v + b.v);
}
inline cdouble operator-(cdouble a, cdouble b) {
    if (!trivial_add(a.v) && !trivial_add(b.v)) n_add++;
    return cdouble(a.v - b.v);
}
inline cdouble operator*(cdouble a, cdouble b) {
    if (!trivial_mul(a.v) && !trivial_mul(b.v)) n_mul++;
    return cdouble(a.v * b.v);
}
inline cdouble operator/(cdouble a, cdouble b) {
    n_div++;
    return cdouble(a.v / b.v);
}
inline cdouble operator-(cdouble a) { return cdouble(-a.v); }
inline cdouble& cdouble::operator+=(cdouble b) { return *this = *this + b; }
inline cdouble& cdouble::operator-=(cdouble b) { return *this = *this - b; }
inline cdouble& cdouble::operator*=(cdouble b) { return *this = *this * b; }
inline cdouble& cdouble::operator/=(cdouble b) { return *this = *this / b; }
inline bool operator<(cdouble a, cdouble b) { return a.v < b.v; }
inline bool operator>(cdouble a, cdouble b) { return a.v > b.v; }
inline bool operator<=(cdouble a, cdouble b) { return a.v <= b.v; }
inline bool operator>=(cdouble a, cdouble b) { return a.v >= b.v; }
inline bool operator==(cdouble a, cdouble b) { return a.v == b.v; }
inline bool operator!=(cdouble a, cdouble b) { return a.v != b.v; }
inline cdouble sqrt(cdouble a) {
    n_sqrt++;
    return cdouble(::sqrt(a.v));
}
inline cdouble fabs(cdouble a) { return cdouble(::fabs(a.v)); }

static_assert(sizeof(cdouble) == sizeof(double), "cdouble must have the layout of double");

#define double cdouble
#include "wb_oracle.c"
#undef double

extern "C" {

void orc_count_reset(void) { n_add = n_mul = n_div = n_sqrt = 0; }

/* out: add/sub, mul, div, sqrt since the last reset */
void orc_count_get(long long out[4])
{
    out[0] = n_add;
    out[1] = n_mul;
    out[2] = n_div;
    out[3] = n_sqrt;
}

}  /* extern "C" */
