/*
 * flopcount.hpp -- a counting double for the oracle's FLOP census.
 *
 * TEST AND MEASUREMENT INFRASTRUCTURE ONLY.  The oracle's C sources are
 * compiled a second time as C++ with `double` replaced by `or_fd`, a struct
 * holding one double (same size, alignment and bit layout, so the oracle's
 * C-ABI structs and arrays are shared unchanged with the plain build).  Every
 * arithmetic operator and math call on an or_fd increments a thread-local
 * counter and computes exactly what the plain double would.
 *
 * Counting rule (the algorithmic work of the method as the oracle writes it
 * out): +, -, *, / and sqrt count one FLOP each; sin, cos, atan2, acos, exp
 * and log count one "special" operation each (reported apart from the FLOPs);
 * comparisons, negation, fabs and copies count nothing.  An operation with an
 * exact-zero operand (x * 0, 0 * x, x + 0, x - 0, 0 - x, 0 / x) is structural:
 * its result is fixed without arithmetic (a zero row of a diagonal block, the
 * unused half of a dense product), so it is not counted.  The census counts
 * the damped linear solves with this rule off (skip_zeros = 0): a solver
 * factors the whole band of its matrix, whatever values it holds.
 */
#ifndef OR_FLOPCOUNT_HPP
#define OR_FLOPCOUNT_HPP

/* Every system header the oracle sources include, included here first so
 * that their declarations keep the real double. */
#include <math.h>
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include <cmath>

struct or_flop_counts {
  int64_t flops;
  int64_t special;
  int skip_zeros; /* 1: operations with an exact-zero operand are not counted */
};
extern thread_local or_flop_counts or_fc;

struct or_fd {
  double v;
  or_fd() = default;
  constexpr or_fd(double x) : v(x) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  or_fd& operator+=(or_fd o);
  or_fd& operator-=(or_fd o);
  or_fd& operator*=(or_fd o);
  or_fd& operator/=(or_fd o);
};

inline void or_fc_add(double a, double b) {
  if (!or_fc.skip_zeros || (a != 0.0 && b != 0.0)) ++or_fc.flops;
}
inline void or_fc_mul(double a, double b) {
  if (!or_fc.skip_zeros || (a != 0.0 && b != 0.0)) ++or_fc.flops;
}
inline or_fd operator+(or_fd a, or_fd b) { or_fc_add(a.v, b.v); return or_fd(a.v + b.v); }
inline or_fd operator-(or_fd a, or_fd b) { or_fc_add(a.v, b.v); return or_fd(a.v - b.v); }
inline or_fd operator*(or_fd a, or_fd b) { or_fc_mul(a.v, b.v); return or_fd(a.v * b.v); }
inline or_fd operator/(or_fd a, or_fd b) {
  if (!or_fc.skip_zeros || a.v != 0.0) ++or_fc.flops;
  return or_fd(a.v / b.v);
}
inline or_fd operator-(or_fd a) { return or_fd(-a.v); }
inline or_fd operator+(or_fd a) { return a; }
inline or_fd& or_fd::operator+=(or_fd o) { *this = *this + o; return *this; }
inline or_fd& or_fd::operator-=(or_fd o) { *this = *this - o; return *this; }
inline or_fd& or_fd::operator*=(or_fd o) { *this = *this * o; return *this; }
inline or_fd& or_fd::operator/=(or_fd o) { *this = *this / o; return *this; }
inline bool operator<(or_fd a, or_fd b) { return a.v < b.v; }
inline bool operator>(or_fd a, or_fd b) { return a.v > b.v; }
inline bool operator<=(or_fd a, or_fd b) { return a.v <= b.v; }
inline bool operator>=(or_fd a, or_fd b) { return a.v >= b.v; }
inline bool operator==(or_fd a, or_fd b) { return a.v == b.v; }
inline bool operator!=(or_fd a, or_fd b) { return a.v != b.v; }
inline bool operator!(or_fd a) { return !a.v; }

inline or_fd sqrt(or_fd a) { ++or_fc.flops; return or_fd(std::sqrt(a.v)); }
inline or_fd fabs(or_fd a) { return or_fd(std::fabs(a.v)); }
inline or_fd sin(or_fd a) { ++or_fc.special; return or_fd(std::sin(a.v)); }
inline or_fd cos(or_fd a) { ++or_fc.special; return or_fd(std::cos(a.v)); }
inline or_fd acos(or_fd a) { ++or_fc.special; return or_fd(std::acos(a.v)); }
inline or_fd exp(or_fd a) { ++or_fc.special; return or_fd(std::exp(a.v)); }
inline or_fd log(or_fd a) { ++or_fc.special; return or_fd(std::log(a.v)); }
inline or_fd atan2(or_fd a, or_fd b) { ++or_fc.special; return or_fd(std::atan2(a.v, b.v)); }
inline bool isfinite(or_fd a) { return std::isfinite(a.v); }
inline bool isnan(or_fd a) { return std::isnan(a.v); }

#endif
