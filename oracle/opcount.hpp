/*
 * opcount.hpp -- an operation-counting stand-in for double, used only to count
 * the floating-point work of the oracle (TEST INFRASTRUCTURE ONLY, like the
 * oracle itself).
 *
 * oracle/opcount.cpp compiles hgks_oracle.c as C++ with every `double`
 * replaced by `opc_double`; each arithmetic operation then adds one to a
 * per-thread counter of its kind before doing the FP64 operation itself, so
 * the oracle computes the same values and reports how many operations of each
 * kind it took.  Counting convention: add / sub, mul, div, sqrt, exp and erfc
 * count one each (and are also tallied by kind); fma counts two; negation,
 * |x|, min / max and comparisons count zero.
 */
#pragma once

#include <cmath>
#include <cstring>

enum { OPC_ADD = 0, OPC_MUL, OPC_FMA, OPC_DIV, OPC_SQRT, OPC_EXP, OPC_ERFC, OPC_KINDS };

extern unsigned long long opc_counts[256][8];
int opc_thread();

#define OPC_TICK(kind) (opc_counts[opc_thread()][kind]++)

struct opc_double {
    double v;
    constexpr opc_double() : v(0.0) {}
    constexpr opc_double(double x) : v(x) {}
    template <class T> explicit operator T() const { return (T)v; }
    opc_double& operator+=(opc_double o) { OPC_TICK(OPC_ADD); v += o.v; return *this; }
    opc_double& operator-=(opc_double o) { OPC_TICK(OPC_ADD); v -= o.v; return *this; }
    opc_double& operator*=(opc_double o) { OPC_TICK(OPC_MUL); v *= o.v; return *this; }
    opc_double& operator/=(opc_double o) { OPC_TICK(OPC_DIV); v /= o.v; return *this; }
};

inline opc_double operator+(opc_double a, opc_double b) { OPC_TICK(OPC_ADD); return opc_double(a.v + b.v); }
inline opc_double operator-(opc_double a, opc_double b) { OPC_TICK(OPC_ADD); return opc_double(a.v - b.v); }
inline opc_double operator*(opc_double a, opc_double b) { OPC_TICK(OPC_MUL); return opc_double(a.v * b.v); }
inline opc_double operator/(opc_double a, opc_double b) { OPC_TICK(OPC_DIV); return opc_double(a.v / b.v); }
inline opc_double operator-(opc_double a) { return opc_double(-a.v); }
inline opc_double operator+(opc_double a) { return a; }
inline bool operator<(opc_double a, opc_double b) { return a.v < b.v; }
inline bool operator>(opc_double a, opc_double b) { return a.v > b.v; }
inline bool operator<=(opc_double a, opc_double b) { return a.v <= b.v; }
inline bool operator>=(opc_double a, opc_double b) { return a.v >= b.v; }
inline bool operator==(opc_double a, opc_double b) { return a.v == b.v; }
inline bool operator!=(opc_double a, opc_double b) { return a.v != b.v; }
inline opc_double fabs(opc_double a) { return opc_double(std::fabs(a.v)); }
inline opc_double fmax(opc_double a, opc_double b) { return opc_double(std::fmax(a.v, b.v)); }
inline opc_double fmin(opc_double a, opc_double b) { return opc_double(std::fmin(a.v, b.v)); }
inline opc_double sqrt(opc_double a) { OPC_TICK(OPC_SQRT); return opc_double(std::sqrt(a.v)); }
inline opc_double exp(opc_double a) { OPC_TICK(OPC_EXP); return opc_double(std::exp(a.v)); }
inline opc_double erfc(opc_double a) { OPC_TICK(OPC_ERFC); return opc_double(std::erfc(a.v)); }
inline opc_double fma(opc_double a, opc_double b, opc_double c) { OPC_TICK(OPC_FMA); return opc_double(std::fma(a.v, b.v, c.v)); }
inline bool isfinite(opc_double a) { return std::isfinite(a.v); }
inline bool isnan(opc_double a) { return std::isnan(a.v); }
