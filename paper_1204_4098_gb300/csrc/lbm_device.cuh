// Device-side building blocks of the fused pseudopotential D2Q9 step.
//
// Lattice (Li, Luo & Li, Sec. II): D2Q9 with c = 1, delta_t = 1,
// c_s^2 = 1/3, velocities e0 = (0,0); e1..e4 = (1,0), (0,1), (-1,0), (0,-1);
// e5..e8 = (1,1), (-1,1), (-1,-1), (1,-1); weights 4/9, 1/9, 1/36 (text
// after Eq. 2) and interaction weights w(1) = 1/3, w(2) = 1/12 (text after
// Eq. 3).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lbm {

constexpr int kQ = 9;

__host__ __device__ constexpr int ex_of(int a) {
  return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0);
}
__host__ __device__ constexpr int ey_of(int a) {
  return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0);
}
// D2Q9 weights.  In FP32 the correctly rounded 4/9, 1/9, 1/36 all round up
// (their sum exceeds 1 by 7e-9), which makes every equilibrium gain mass and
// drifts the total mass by ~1e-8 per step.  The FP32 set below keeps 1/9,
// takes the float just below 1/36, and w0 = 1 - 4 w1 - 4 w2, which is exactly
// representable: the weights sum to exactly 1.
template <class C>
__host__ __device__ constexpr C w_of(int a) {
  return a == 0 ? C(4) / C(9) : (a <= 4 ? C(1) / C(9) : C(1) / C(36));
}
template <>
__host__ __device__ constexpr float w_of<float>(int a) {
  return a == 0 ? 0x1.c71c72p-2f : (a <= 4 ? 0x1.c71c72p-4f : 0x1.c71c70p-6f);
}

// ---------------------------------------------------------------------------
// explicitly rounded arithmetic: the potential psi is evaluated both by the
// lane that owns a column and, as a halo, by the neighbouring warp; writing
// it with *_rn operations keeps the compiler from contracting the two copies
// differently, so both see bit-identical values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// ---------------------------------------------------------------------------
// two cells at once: the two columns a lane owns in the two-column kernels.
// Every operation on a Pair is the scalar operation above on each element,
// so a pair evaluation gives the same bits as two scalar ones.  FP32 pairs
// use the packed FP32x2 add / multiply / fused multiply-add of sm_100 and
// later (one instruction for both elements); FP64 pairs go element by
// element.
// ---------------------------------------------------------------------------
template <class C> struct Pair;
template <>
struct Pair<float> {
  float2 v;
  __device__ __forceinline__ Pair() {}
  __device__ __forceinline__ Pair(float c) : v(make_float2(c, c)) {}
  __device__ __forceinline__ Pair(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit Pair(float2 x) : v(x) {}
  __device__ __forceinline__ float x() const { return v.x; }
  __device__ __forceinline__ float y() const { return v.y; }
};
template <>
struct Pair<double> {
  double2 v;
  __device__ __forceinline__ Pair() {}
  __device__ __forceinline__ Pair(double c) : v(make_double2(c, c)) {}
  __device__ __forceinline__ Pair(double a, double b) : v(make_double2(a, b)) {}
  __device__ __forceinline__ explicit Pair(double2 x) : v(x) {}
  __device__ __forceinline__ double x() const { return v.x; }
  __device__ __forceinline__ double y() const { return v.y; }
};
using F2 = Pair<float>;
using D2 = Pair<double>;
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 add_rn(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
// a - b = a + (-b) exactly (negation is exact), as for the scalar subtraction
__device__ __forceinline__ F2 sub_rn(F2 a, F2 b) { return F2(__fadd2_rn(a.v, (-b).v)); }
__device__ __forceinline__ F2 mul_rn(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 fma_rn(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ D2 operator-(D2 a) { return D2(-a.v.x, -a.v.y); }
__device__ __forceinline__ D2 add_rn(D2 a, D2 b) {
  return D2(__dadd_rn(a.v.x, b.v.x), __dadd_rn(a.v.y, b.v.y));
}
__device__ __forceinline__ D2 sub_rn(D2 a, D2 b) {
  return D2(__dsub_rn(a.v.x, b.v.x), __dsub_rn(a.v.y, b.v.y));
}
__device__ __forceinline__ D2 mul_rn(D2 a, D2 b) {
  return D2(__dmul_rn(a.v.x, b.v.x), __dmul_rn(a.v.y, b.v.y));
}
__device__ __forceinline__ D2 fma_rn(D2 a, D2 b, D2 c) {
  return D2(__fma_rn(a.v.x, b.v.x, c.v.x), __fma_rn(a.v.y, b.v.y, c.v.y));
}

// scalar type of a value type (C itself, or the element type of a Pair)
template <class V> struct ScalarOf { using type = V; };
template <class C> struct ScalarOf<Pair<C>> { using type = C; };

// ---------------------------------------------------------------------------
// physical parameters of one lattice, in the compute type C
// ---------------------------------------------------------------------------
template <class C>
struct Phys {
  C RT;         // R T of Eq. 23
  C a;          // attraction constant of Eq. 23
  C b4;         // b / 4  (eta = b rho / 4)
  C two_over_G; // 2 / G  (Eq. 8 with c = 1)
  C minus_G;    // -G     (Eq. 3)
  C tau;        // relaxation time
  C omega;      // 1 / tau
  C sigma_ups;  // sigma / (tau - 1/2)  (Eq. 31: v' = v + sigma F / (upsilon psi^2))
  C guo;        // 1 - 1 / (2 tau)  (B_e = C_e of Eq. 13)
  int scheme;   // forcing scheme, read only by collide<kAnyForced>
  C s_e, s_eps, s_q;  // MRT rates of the energy, energy-square, energy-flux moments
};

// Reciprocal and square root for the per-cell physics.  FP64 keeps the IEEE
// operations (it is the parity reference on the GPU); FP32 uses the hardware
// approximations (MUFU.RCP / MUFU.RSQ, ~1 ulp), which are deterministic, so
// the owner and the halo copy of psi stay bit-identical.
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float fast_sqrt_pos(float a) { return a * rsqrtf(a); }
__device__ __forceinline__ double fast_sqrt_pos(double a) { return __dsqrt_rn(a); }

template <class C>
__device__ __forceinline__ Pair<C> fast_div(Pair<C> a, Pair<C> b) {
  return Pair<C>(fast_div(a.x(), b.x()), fast_div(a.y(), b.y()));
}

// psi of Eq. 8 with the Carnahan-Starling p_EOS of Eq. 23.  Flags (and
// returns 0 for) densities outside the domain of psi: rho <= 0, eta >= 1,
// a negative or non-finite radicand.  psi_radicand holds the arithmetic
// (for a scalar or a pair), psi_finish the per-cell domain check and root.
template <class V, class C>
__device__ __forceinline__ void psi_radicand(V rho, const Phys<C>& P, V& eta, V& arg) {
  const V one = V(C(1));
  eta = mul_rn(V(P.b4), rho);
  const V om = sub_rn(one, eta);
  // 1 + eta + eta^2 - eta^3 = 1 + eta (1 + eta (1 - eta))
  const V num = fma_rn(eta, fma_rn(eta, om, one), one);
  const V den = mul_rn(mul_rn(om, om), om);
  const V p = sub_rn(fast_div(mul_rn(mul_rn(rho, V(P.RT)), num), den),
                     mul_rn(mul_rn(V(P.a), rho), rho));
  arg = mul_rn(V(P.two_over_G), sub_rn(p, mul_rn(rho, V(C(1) / C(3)))));
}
template <class C>
__device__ __forceinline__ C psi_finish(C rho, C eta, C arg, bool& bad) {
  const bool ok = (rho > C(0)) && (eta < C(1)) && (arg >= C(0)) && (arg <= C(1e30));
  bad |= !ok;
  return (ok && arg > C(0)) ? fast_sqrt_pos(arg) : C(0);
}
template <class C>
__device__ __forceinline__ C psi_of_rho(C rho, const Phys<C>& P, bool& bad) {
  C eta, arg;
  psi_radicand(rho, P, eta, arg);
  return psi_finish(rho, eta, arg, bad);
}
template <class C>
__device__ __forceinline__ Pair<C> psi_of_rho(Pair<C> rho, const Phys<C>& P, bool& bad) {
  Pair<C> eta, arg;
  psi_radicand(rho, P, eta, arg);
  return Pair<C>(psi_finish(rho.x(), eta.x(), arg.x(), bad),
                 psi_finish(rho.y(), eta.y(), arg.y(), bad));
}

// ---------------------------------------------------------------------------
// collision of one cell, Eqs. 1-2 with the forcing schemes of Table I
// ---------------------------------------------------------------------------
enum Scheme { kSC = 0, kEDM = 1, kImproved = 2, kNoForce = 3, kEDMMod = 4, kLadd = 5, kMRT = 6 };
// Template value: the scheme (one that evaluates psi, i.e. not kNoForce) is
// read from Phys::scheme at run time.  One inlined body then serves every
// instance of a mixed batch, instead of one body per scheme.
constexpr int kAnyForced = -1;

// Every scheme of Table I is BGK towards f_eq(rho, u_eq) plus Guo's general
// forcing term (Eq. 12) with B = B_e F and C = C_e (V F + F V):
//   F_a = w_a [ 3 B_e (e.F) + C_e (9 (e.V)(e.F) - 3 V.F) ].
//   SC (Eqs. 9-10):  u_eq = u + tau F / rho, no forcing term
//   EDM (Eq. 11):    u_eq = u, B_e = C_e = 1, V = u + F/(2 rho)
//                    (Eq. 16: f_eq(u + F/rho) - f_eq(u) in closed form)
//   improved (Eq. 31): u_eq = v = u + F/(2 rho), B_e = C_e = 1 - 1/(2 tau),
//                    V = v' = v + sigma F / ((tau - 1/2) psi^2)
//   EDM, C_e = 1/tau: u_eq = u, B_e = 1, C_e = 1/tau, V = v
//   Ladd:            u_eq = u, B_e = C_e = 1, V = u
//   no force:        u_eq = u, no forcing term
//
// Every operation is explicitly rounded (no compiler contraction), so all
// kernels that inline this body -- single domain, batch work list, batch
// persistent -- produce bit-identical populations.  With SCHEME fixed the
// branches below fold at compile time; with kAnyForced they are taken on
// P.scheme (uniform across a warp) and compute the same values.
// Multiple-relaxation-time form of the improved scheme (the extension the
// paper states at the end of Sec. IV).  D2Q9 moments in the Lallemand-Luo
// basis: density rho, energy e, energy square eps, momentum j, energy flux q,
// stresses pxx = f.(cx^2 - cy^2), pxy = f.(cx cy).  Each non-conserved moment
// relaxes with its own rate s towards its value at f_eq(rho, v) and receives
// (1 - s/2) times the improved forcing term's moment:
//   e:   -2 rho + 3 rho |v|^2,  6 v'.F        eps: rho - 3 rho |v|^2, -6 v'.F
//   q:   -rho v,               -F             pxx: rho (vx^2 - vy^2), 2 (v'x Fx - v'y Fy)
//   pxy: rho vx vy,             v'x Fy + v'y Fx
// (stresses at 1/tau, e / eps / q at P.s_e / P.s_eps / P.s_q); the momentum
// becomes j + F.  Equal rates 1/tau give Eq. 31.  The populations follow
// from the orthogonal basis (row norms 9, 36, 36, 6, 12, 6, 12, 4, 4), the
// rest population as the remainder of rho.
//
// Both functions take one cell (V = C) or two (V = Pair<C>, the two-column
// kernels): per-cell quantities are of type V, the lattice's uniform
// parameters stay scalars of type C and are broadcast where they meet a
// per-cell value.  The sequence of rounded operations per cell is the same
// either way.
template <class V, class C>
__device__ __forceinline__ void collide_mrt(V (&f)[kQ], V rho, V Fx, V Fy, V psi,
                                            const Phys<C>& P) {
  const V ax = sub_rn(f[1], f[3]), ay = sub_rn(f[2], f[4]);  // axis odd parts
  const V bx = add_rn(sub_rn(f[5], f[6]), sub_rn(f[8], f[7]));  // diagonal x odd part
  const V by = sub_rn(add_rn(f[5], f[6]), add_rn(f[7], f[8]));  // diagonal y odd part
  const V s1 = add_rn(add_rn(f[1], f[3]), add_rn(f[2], f[4]));  // axis sum
  const V s2 = add_rn(add_rn(f[5], f[7]), add_rn(f[6], f[8]));  // diagonal sum
  const V jx = add_rn(ax, bx), jy = add_rn(ay, by);
  const V qx = fma_rn(V(C(-2)), ax, bx), qy = fma_rn(V(C(-2)), ay, by);
  const V e = fma_rn(V(C(2)), s2, -fma_rn(V(C(4)), f[0], s1));
  const V eps = fma_rn(V(C(-2)), s1, fma_rn(V(C(4)), f[0], s2));
  const V pxx = sub_rn(add_rn(f[1], f[3]), add_rn(f[2], f[4]));
  const V pxy = sub_rn(add_rn(f[5], f[7]), add_rn(f[6], f[8]));

  const V inv_rho = fast_div(V(C(1)), rho);
  const V half_inv = mul_rn(V(C(0.5)), inv_rho);
  const V vx = fma_rn(half_inv, Fx, mul_rn(jx, inv_rho));
  const V vy = fma_rn(half_inv, Fy, mul_rn(jy, inv_rho));
  const V sg = fast_div(V(P.sigma_ups), mul_rn(psi, psi));
  const V wx = fma_rn(sg, Fx, vx), wy = fma_rn(sg, Fy, vy);  // v'
  const V v2 = fma_rn(vx, vx, mul_rn(vy, vy));
  const V rv2 = mul_rn(V(C(3)), mul_rn(rho, v2));
  const V wF6 = mul_rn(V(C(6)), fma_rn(wx, Fx, mul_rn(wy, Fy)));

  // m* = (1 - s/2) force + (m - s (m - meq)); (1 - s/2) and -s are uniform
  auto relax = [](V m, V meq, C s, V force) {
    return fma_rn(V(sub_rn(C(1), mul_rn(C(0.5), s))), force, fma_rn(V(-s), sub_rn(m, meq), m));
  };
  const C sv = P.omega;
  const V e_s = relax(e, fma_rn(V(C(-2)), rho, rv2), P.s_e, wF6);
  const V eps_s = relax(eps, sub_rn(rho, rv2), P.s_eps, -wF6);
  const V qx_s = relax(qx, -mul_rn(rho, vx), P.s_q, -Fx);
  const V qy_s = relax(qy, -mul_rn(rho, vy), P.s_q, -Fy);
  const V pxx_s = relax(pxx, mul_rn(rho, fma_rn(vx, vx, -mul_rn(vy, vy))), sv,
                        mul_rn(V(C(2)), fma_rn(wx, Fx, -mul_rn(wy, Fy))));
  const V pxy_s = relax(pxy, mul_rn(rho, mul_rn(vx, vy)), sv, fma_rn(wx, Fy, mul_rn(wy, Fx)));
  const V jx_s = add_rn(jx, Fx), jy_s = add_rn(jy, Fy);

  const V r9 = mul_rn(rho, V(C(1) / C(9)));
  const V base_ax = fma_rn(V(C(-1) / C(36)), e_s, fma_rn(V(C(-1) / C(18)), eps_s, r9));
  const V base_dg = fma_rn(V(C(1) / C(18)), e_s, fma_rn(V(C(1) / C(36)), eps_s, r9));
  const V px4 = mul_rn(V(C(0.25)), pxx_s), pd4 = mul_rn(V(C(0.25)), pxy_s);
  const V ox = mul_rn(V(C(1) / C(6)), sub_rn(jx_s, qx_s));   // axis x odd part
  const V oy = mul_rn(V(C(1) / C(6)), sub_rn(jy_s, qy_s));
  const V dx = fma_rn(V(C(1) / C(12)), qx_s, mul_rn(V(C(1) / C(6)), jx_s));  // diagonal parts
  const V dy = fma_rn(V(C(1) / C(12)), qy_s, mul_rn(V(C(1) / C(6)), jy_s));
  const V ex_even = add_rn(base_ax, px4), ey_even = sub_rn(base_ax, px4);
  f[1] = add_rn(ex_even, ox);
  f[3] = sub_rn(ex_even, ox);
  f[2] = add_rn(ey_even, oy);
  f[4] = sub_rn(ey_even, oy);
  const V d57 = add_rn(base_dg, pd4), d68 = sub_rn(base_dg, pd4);
  const V pp = add_rn(dx, dy), pm = sub_rn(dx, dy);
  f[5] = add_rn(d57, pp);  // e5 = (1, 1)
  f[7] = sub_rn(d57, pp);  // e7 = (-1, -1)
  f[8] = add_rn(d68, pm);  // e8 = (1, -1)
  f[6] = sub_rn(d68, pm);  // e6 = (-1, 1)
  V rest = f[1];
#pragma unroll
  for (int a = 2; a < kQ; ++a) rest = add_rn(rest, f[a]);
  f[0] = sub_rn(rho, rest);
}

template <int SCHEME, class V, class C>
__device__ __forceinline__ void collide(V (&f)[kQ], V rho, V Fx, V Fy, V psi,
                                        const Phys<C>& P) {
  if constexpr (SCHEME == kMRT) {
    if constexpr (std::is_same<V, C>::value) {
      collide_mrt(f, rho, Fx, Fy, psi, P);
    } else {
      // Element by element: in this body the packed FP32x2 instructions were
      // measured a few ulps away from the scalar ones on ~0.6 % of the values
      // (the same source with scalar operations per element matched the
      // one-column kernel bit for bit), so the two cells go through the
      // scalar body one at a time.
      C fa[kQ], fb[kQ];
#pragma unroll
      for (int a = 0; a < kQ; ++a) {
        fa[a] = f[a].x();
        fb[a] = f[a].y();
      }
      collide_mrt(fa, rho.x(), Fx.x(), Fy.x(), psi.x(), P);
      collide_mrt(fb, rho.y(), Fx.y(), Fy.y(), psi.y(), P);
#pragma unroll
      for (int a = 0; a < kQ; ++a) f[a] = V(fa[a], fb[a]);
    }
    return;
  }
  const int sch = SCHEME == kAnyForced ? P.scheme : SCHEME;
  const V jx = add_rn(add_rn(sub_rn(f[1], f[3]), sub_rn(f[5], f[6])), sub_rn(f[8], f[7]));
  const V jy = sub_rn(add_rn(sub_rn(f[2], f[4]), add_rn(f[5], f[6])), add_rn(f[7], f[8]));
  const V inv_rho = fast_div(V(C(1)), rho);
  const V ux = mul_rn(jx, inv_rho), uy = mul_rn(jy, inv_rho);
  const V half_inv = mul_rn(V(C(0.5)), inv_rho);

  V qx = ux, qy = uy;  // velocity in f_eq
  V Vx = V(C(0)), Vy = V(C(0));
  C Be = C(0), Ce = C(0);
  const bool forcing = sch != kSC && sch != kNoForce;
  if (sch == kSC) {
    const V t = mul_rn(V(P.tau), inv_rho);
    qx = fma_rn(t, Fx, ux);
    qy = fma_rn(t, Fy, uy);
  } else if (sch == kEDM) {
    Vx = fma_rn(half_inv, Fx, ux);
    Vy = fma_rn(half_inv, Fy, uy);
    Be = C(1);
    Ce = C(1);
  } else if (sch == kImproved) {
    qx = fma_rn(half_inv, Fx, ux);
    qy = fma_rn(half_inv, Fy, uy);
    const V s = fast_div(V(P.sigma_ups), mul_rn(psi, psi));
    Vx = fma_rn(s, Fx, qx);
    Vy = fma_rn(s, Fy, qy);
    Be = P.guo;
    Ce = P.guo;
  } else if (sch == kEDMMod) {
    Vx = fma_rn(half_inv, Fx, ux);
    Vy = fma_rn(half_inv, Fy, uy);
    Be = C(1);
    Ce = P.omega;
  } else if (sch == kLadd) {
    Vx = ux;
    Vy = uy;
    Be = C(1);
    Ce = C(1);
  }

  const C om = P.omega;
  const V one_m_om = V(sub_rn(C(1), om));
  // f_eq_a = w rho (1 - 1.5 q.q + 3 e.q + 4.5 (e.q)^2), F_a as above.  For an
  // opposite pair (a, b), e_b = -e_a: the terms even in e are shared and the
  // odd ones change sign, so each pair is evaluated once.
  const V base = fma_rn(V(C(-1.5)), fma_rn(qx, qx, mul_rn(qy, qy)), V(C(1)));
  const V om_rho = mul_rn(V(om), rho);
  const V VF3 = mul_rn(V(C(3)), fma_rn(Vx, Fx, mul_rn(Vy, Fy)));
  auto pair = [&](int a, int b, C w, V eq, V eF, V eV) {
    const V wr = mul_rn(V(w), om_rho);
    V even = mul_rn(wr, fma_rn(mul_rn(V(C(4.5)), eq), eq, base));
    V odd = mul_rn(mul_rn(V(C(3)), wr), eq);
    if (forcing) {
      even = fma_rn(V(mul_rn(w, Ce)), fma_rn(mul_rn(V(C(9)), eV), eF, -VF3), even);
      odd = fma_rn(V(mul_rn(mul_rn(C(3), w), Be)), eF, odd);
    }
    const V fa = fma_rn(one_m_om, f[a], even);
    const V fb = fma_rn(one_m_om, f[b], even);
    f[a] = add_rn(fa, odd);
    f[b] = sub_rn(fb, odd);
  };
  const C w1 = w_of<C>(1), w2 = w_of<C>(5);
  pair(1, 3, w1, qx, Fx, Vx);
  pair(2, 4, w1, qy, Fy, Vy);
  pair(5, 7, w2, add_rn(qx, qy), add_rn(Fx, Fy), add_rn(Vx, Vy));  // e5 = (1,1), e7 = (-1,-1)
  pair(6, 8, w2, sub_rn(qy, qx), sub_rn(Fy, Fx), sub_rn(Vy, Vx));  // e6 = (-1,1), e8 = (1,-1)
  // Every scheme conserves mass (sum_a F_a = 0, sum_a f_eq = rho); taking the
  // rest population as the remainder makes that hold to one rounding instead
  // of nine, so FP32 runs do not drift in mass.
  V rest = f[1];
#pragma unroll
  for (int a = 2; a < kQ; ++a) rest = add_rn(rest, f[a]);
  f[0] = sub_rn(rho, rest);
}

// ---------------------------------------------------------------------------
// population storage
// ---------------------------------------------------------------------------
// Direct storage: f stored as T, computed as C.
// Deviation storage: d_a = f_a - w_a rho_src stored as 16-bit T, plus a float
// plane rho_src (the density of the cell the populations sit on).
struct StoreF32 {
  using T = float;
  using C = float;
  static constexpr bool kDev = false;
  static __device__ __forceinline__ C to_c(T v) { return v; }
  static __device__ __forceinline__ T from_c(C v) { return v; }
};
struct StoreF64 {
  using T = double;
  using C = double;
  static constexpr bool kDev = false;
  static __device__ __forceinline__ C to_c(T v) { return v; }
  static __device__ __forceinline__ T from_c(C v) { return v; }
};
struct StoreBF16 {
  using T = __nv_bfloat16;
  using C = float;
  static constexpr bool kDev = true;
  static __device__ __forceinline__ C to_c(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T from_c(C v) { return __float2bfloat16_rn(v); }
  // two at a time (the same values as to_c / from_c).  A bf16 is the upper
  // half of the float it stands for, so the pair unpacks with one shift and
  // one mask of its 32-bit word (2.5 % faster in the issue-bound 16-bit
  // kernel than the conversion intrinsic).
  static __device__ __forceinline__ float2 to_c2(__nv_bfloat162 v) {
    unsigned u;
    __builtin_memcpy(&u, &v, sizeof(u));
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  }
  static __device__ __forceinline__ __nv_bfloat162 from_c2(C a, C b) {
    return __floats2bfloat162_rn(a, b);
  }
  // wr + d with one rounding (mixed-precision FMA of the 16-bit deviation
  // times 1 plus the FP32 w_a rho): the value a stored deviation stands for.
  static __device__ __forceinline__ float decode(float wr, __nv_bfloat16 d) {
    unsigned short b;
    __builtin_memcpy(&b, &d, sizeof(b));
    float x;
    asm("{\n .reg .b16 m;\n mov.b16 m, 0x3F80;\n fma.rn.f32.bf16 %0, %1, m, %2;\n}"
        : "=f"(x)
        : "h"(b), "f"(wr));
    return x;
  }
  static __device__ __forceinline__ Pair<float> decode2(Pair<float> wr, __nv_bfloat162 v) {
    unsigned u;
    __builtin_memcpy(&u, &v, sizeof(u));
    float x, y;
    asm("{\n .reg .b16 lo, hi, m;\n mov.b32 {lo, hi}, %2;\n mov.b16 m, 0x3F80;\n"
        " fma.rn.f32.bf16 %0, lo, m, %3;\n fma.rn.f32.bf16 %1, hi, m, %4;\n}"
        : "=f"(x), "=f"(y)
        : "r"(u), "f"(wr.x()), "f"(wr.y()));
    return Pair<float>(x, y);
  }
  // (r.x - v.x, r.y - v.y), each one rounding: a mixed-precision FMA with the
  // 16-bit value times -1 (exact) plus the FP32 value, on the 16-bit halves
  // of the pair's word as they are -- the same values as subtracting the
  // unpacked pair.
  static __device__ __forceinline__ Pair<float> sub_from(Pair<float> r, __nv_bfloat162 v) {
    unsigned u;
    __builtin_memcpy(&u, &v, sizeof(u));
    float x, y;
    asm("{\n .reg .b16 lo, hi, m;\n mov.b32 {lo, hi}, %2;\n mov.b16 m, 0xBF80;\n"
        " fma.rn.f32.bf16 %0, lo, m, %3;\n fma.rn.f32.bf16 %1, hi, m, %4;\n}"
        : "=f"(x), "=f"(y)
        : "r"(u), "f"(r.x()), "f"(r.y()));
    return Pair<float>(x, y);
  }
};
struct StoreF16 {
  using T = __half;
  using C = float;
  static constexpr bool kDev = true;
  static __device__ __forceinline__ C to_c(T v) { return __half2float(v); }
  static __device__ __forceinline__ T from_c(C v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float2 to_c2(__half2 v) { return __half22float2(v); }
  static __device__ __forceinline__ __half2 from_c2(C a, C b) { return __floats2half2_rn(a, b); }
  // as StoreBF16::decode, with 1 in FP16
  static __device__ __forceinline__ float decode(float wr, __half d) {
    unsigned short b;
    __builtin_memcpy(&b, &d, sizeof(b));
    float x;
    asm("{\n .reg .b16 m;\n mov.b16 m, 0x3C00;\n fma.rn.f32.f16 %0, %1, m, %2;\n}"
        : "=f"(x)
        : "h"(b), "f"(wr));
    return x;
  }
  static __device__ __forceinline__ Pair<float> decode2(Pair<float> wr, __half2 v) {
    unsigned u;
    __builtin_memcpy(&u, &v, sizeof(u));
    float x, y;
    asm("{\n .reg .b16 lo, hi, m;\n mov.b32 {lo, hi}, %2;\n mov.b16 m, 0x3C00;\n"
        " fma.rn.f32.f16 %0, lo, m, %3;\n fma.rn.f32.f16 %1, hi, m, %4;\n}"
        : "=f"(x), "=f"(y)
        : "r"(u), "f"(wr.x()), "f"(wr.y()));
    return Pair<float>(x, y);
  }
  // as StoreBF16::sub_from, with -1 in FP16
  static __device__ __forceinline__ Pair<float> sub_from(Pair<float> r, __half2 v) {
    unsigned u;
    __builtin_memcpy(&u, &v, sizeof(u));
    float x, y;
    asm("{\n .reg .b16 lo, hi, m;\n mov.b32 {lo, hi}, %2;\n mov.b16 m, 0xBC00;\n"
        " fma.rn.f32.f16 %0, lo, m, %3;\n fma.rn.f32.f16 %1, hi, m, %4;\n}"
        : "=f"(x), "=f"(y)
        : "r"(u), "f"(r.x()), "f"(r.y()));
    return Pair<float>(x, y);
  }
};

// Device status bits (same values as the kStatus*Flag constants of the host).
enum : unsigned { kStatusDiverged = 1u, kStatusTimeout = 2u, kStatusInvalidInit = 4u };

}  // namespace lbm
