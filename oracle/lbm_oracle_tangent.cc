/*
 * Tangent (forward-mode derivative) of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY, like lbm_oracle.c: used by the tests to check
 * the CUDA library's discrete adjoint against the oracle's own derivative.
 * It shares no code with the CUDA library.
 *
 * This file compiles lbm_oracle.c unchanged, as C++, with its arithmetic
 * type `real` a dual number (v, d): v follows the oracle's double-precision
 * arithmetic operation by operation, and d is the derivative of v along one
 * direction of the inputs (state, material fields, operating parameters),
 * carried by the chain rule through every operation.  One run of the step
 * therefore gives the step's value and its Jacobian-vector product J w.
 * The rules are the textbook derivatives of + - * /, sqrt, exp, pow and
 * |.|; comparisons and branches use the values, as the oracle does.
 *
 * |v| has no derivative at v = 0 (a velocity at rest); the oracle uses it
 * only inside Eq. 8's u = v / den(|v|) and in the Forchheimer term
 * |u| u, both differentiable there with a derivative that does not involve
 * d|v|.  sqrt therefore takes derivative 0 at 0, the one value that keeps
 * those compositions exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

struct dual {
  double v, d;
  dual() = default;
  constexpr dual(double x) : v(x), d(0.0) {}
  constexpr dual(double x, double dx) : v(x), d(dx) {}
  dual &operator+=(const dual &b) { d += b.d; v += b.v; return *this; }
  dual &operator-=(const dual &b) { d -= b.d; v -= b.v; return *this; }
  dual &operator*=(const dual &b) { d = d * b.v + v * b.d; v *= b.v; return *this; }
  dual &operator/=(const dual &b) {
    const double q = v / b.v;
    d = (d - q * b.d) / b.v;
    v = q;
    return *this;
  }
};
static inline dual operator-(const dual &a) { return dual(-a.v, -a.d); }
static inline dual operator+(const dual &a, const dual &b) { return dual(a.v + b.v, a.d + b.d); }
static inline dual operator-(const dual &a, const dual &b) { return dual(a.v - b.v, a.d - b.d); }
static inline dual operator*(const dual &a, const dual &b) {
  return dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
static inline dual operator/(const dual &a, const dual &b) {
  const double q = a.v / b.v;
  return dual(q, (a.d - q * b.d) / b.v);
}
static inline dual operator+(double a, const dual &b) { return dual(a) + b; }
static inline dual operator+(const dual &a, double b) { return a + dual(b); }
static inline dual operator-(double a, const dual &b) { return dual(a) - b; }
static inline dual operator-(const dual &a, double b) { return a - dual(b); }
static inline dual operator*(double a, const dual &b) { return dual(a * b.v, a * b.d); }
static inline dual operator*(const dual &a, double b) { return dual(a.v * b, a.d * b); }
static inline dual operator/(double a, const dual &b) { return dual(a) / b; }
static inline dual operator/(const dual &a, double b) { return dual(a.v / b, a.d / b); }
static inline bool operator<(const dual &a, const dual &b) { return a.v < b.v; }
static inline bool operator>(const dual &a, const dual &b) { return a.v > b.v; }
static inline bool operator<=(const dual &a, const dual &b) { return a.v <= b.v; }
static inline bool operator>=(const dual &a, const dual &b) { return a.v >= b.v; }
static inline bool operator==(const dual &a, const dual &b) { return a.v == b.v; }
static inline bool operator!=(const dual &a, const dual &b) { return a.v != b.v; }
static inline bool operator<(const dual &a, double b) { return a.v < b; }
static inline bool operator>(const dual &a, double b) { return a.v > b; }
static inline bool operator<(double a, const dual &b) { return a < b.v; }
static inline bool operator>(double a, const dual &b) { return a > b.v; }

static inline dual sqrt(const dual &a) {
  const double r = sqrt(a.v);
  return dual(r, r > 0.0 ? a.d / (2.0 * r) : 0.0);
}
static inline dual exp(const dual &a) {
  const double e = exp(a.v);
  return dual(e, e * a.d);
}
static inline dual pow(const dual &a, double p) {
  return dual(pow(a.v, p), p * pow(a.v, p - 1.0) * a.d);
}
static inline dual fabs(const dual &a) { return a.v < 0.0 ? -a : a; }
static inline bool isinf(const dual &a) { return isinf(a.v); }
static inline bool isnan(const dual &a) { return isnan(a.v); }

#define ORC_REAL_DEFINED
typedef dual real;

extern "C" {
#include "lbm_oracle.c"
}
