// Pointwise ideal-MHD physics on the device (one thread = one point).
//
// Conserved variables u = (rho, m_x, m_y, m_z, E, B_x, B_y, B_z[, psi]) (Sec. 2).
// * flux_dir: analytic flux of eq. mhd-flux along axis a; GLM adds psi to the
//   B_a row and c_h^2 B_a as the psi flux (Sec. 4.1.5);
// * bn_face: eq. bxface-average-alfven;
// * glm_face: upwinded (B_n*, psi*) of the linear GLM subsystem (Sec. 4.1.5);
// * hlld: Miyoshi & Kusano (2005) five-wave flux, the solver of Sec. 4.1.2,
//   with the normal field of both states set to B^n_F first (Sec. 4.1.3), the
//   thermal pressure of each state kept.
#pragma once
#include <cuda_runtime.h>

namespace dgmhd {

template <typename T>
__device__ __forceinline__ T dsqrt(T x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

// Reciprocals and quotients: exact IEEE operations in FP64; in FP32 the fast
// hardware reciprocal forms (__fdividef, rsqrtf: a few ulp), far inside the
// FP32 form's tolerance and a fraction of the instructions of an IEEE division.
template <typename T>
__device__ __forceinline__ T rcp(T x) { return T(1) / x; }
template <>
__device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.f, x); }
template <typename T>
__device__ __forceinline__ T quot(T a, T b) { return a / b; }
template <>
__device__ __forceinline__ float quot<float>(float a, float b) { return __fdividef(a, b); }
template <typename T>
__device__ __forceinline__ T rsq(T x) { return T(1) / sqrt(x); }
template <>
__device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }

template <typename T>
__device__ __forceinline__ void flux_dir(const T* u, int a, T gamma, bool glm, T ch2, T* f) {
  const T rho = u[0];
  const T ir = rcp(rho);
  const T vx = u[1] * ir, vy = u[2] * ir, vz = u[3] * ir;
  const T bx = u[5], by = u[6], bz = u[7];
  const T b2 = bx * bx + by * by + bz * bz;
  const T p = (gamma - T(1)) * (u[4] - T(0.5) * rho * (vx * vx + vy * vy + vz * vz) - T(0.5) * b2);
  const T pT = p + T(0.5) * b2;
  const T va = a == 0 ? vx : (a == 1 ? vy : vz);
  const T ba = a == 0 ? bx : (a == 1 ? by : bz);
  const T vb = vx * bx + vy * by + vz * bz;
  f[0] = u[1 + a];
  f[1] = u[1] * va - bx * ba;
  f[2] = u[2] * va - by * ba;
  f[3] = u[3] * va - bz * ba;
  f[1 + a] += pT;
  f[4] = (u[4] + pT) * va - vb * ba;
  f[5] = bx * va - vx * ba;
  f[6] = by * va - vy * ba;
  f[7] = bz * va - vz * ba;
  if (glm) {
    f[5 + a] += u[8];
    f[8] = ch2 * ba;
  }
}

template <typename T>
__device__ __forceinline__ T bn_face(T rL, T rR, T bL, T bR) {
  const T sL = rsq(rL), sR = rsq(rR);
  return quot(bL * sL + bR * sR, sL + sR);
}

// Rotated-frame state: rho, u (normal), v, w (tangential), p, By, Bz (tangential)
template <typename T>
struct Prim {
  T r, u, v, w, p, by, bz;
};

// HLLD flux in the rotated frame; out[0..7] = (rho, m_n, m_t1, m_t2, E, B_n, B_t1, B_t2).
// st (nullable): velocity (u, v, w) and tangential field (by, bz) of the
// interface state, the state of the Riemann fan that contains the face
// (Sec. 4.1.3, "Interface state"); its normal field is bn.
template <typename T>
__device__ __forceinline__ void hlld(const Prim<T>& L, const Prim<T>& R, T bn, T gamma, T eps, T* out,
                                     Prim<T>* st = nullptr) {
  auto set_state = [&](T u, T v, T w, T by, T bz) {
    if (st) {
      st->u = u; st->v = v; st->w = w; st->by = by; st->bz = bz;
    }
  };
  const T gm1i = rcp(gamma - T(1));
  const T bn2 = bn * bn;
  const T b2L = bn2 + L.by * L.by + L.bz * L.bz;
  const T b2R = bn2 + R.by * R.by + R.bz * R.bz;
  const T EL = L.p * gm1i + T(0.5) * L.r * (L.u * L.u + L.v * L.v + L.w * L.w) + T(0.5) * b2L;
  const T ER = R.p * gm1i + T(0.5) * R.r * (R.u * R.u + R.v * R.v + R.w * R.w) + T(0.5) * b2R;
  const T pTL = L.p + T(0.5) * b2L, pTR = R.p + T(0.5) * b2R;
  // fast speeds
  T cfL, cfR;
  {
    const T irL = rcp(L.r), irR = rcp(R.r);
    T a2 = gamma * L.p * irL, bb = b2L * irL, bn2r = bn2 * irL;
    T disc = (a2 + bb) * (a2 + bb) - T(4) * a2 * bn2r;
    disc = disc > T(0) ? disc : T(0);
    cfL = dsqrt(T(0.5) * (a2 + bb + dsqrt(disc)));
    a2 = gamma * R.p * irR;
    bb = b2R * irR;
    bn2r = bn2 * irR;
    disc = (a2 + bb) * (a2 + bb) - T(4) * a2 * bn2r;
    disc = disc > T(0) ? disc : T(0);
    cfR = dsqrt(T(0.5) * (a2 + bb + dsqrt(disc)));
  }
  const T cmax = cfL > cfR ? cfL : cfR;
  const T SL = (L.u < R.u ? L.u : R.u) - cmax;
  const T SR = (L.u > R.u ? L.u : R.u) + cmax;

  auto phys = [&](const Prim<T>& s, T E, T pT, T* F, T* U) {
    const T vb = s.u * bn + s.v * s.by + s.w * s.bz;
    U[0] = s.r; U[1] = s.r * s.u; U[2] = s.r * s.v; U[3] = s.r * s.w;
    U[4] = E; U[5] = bn; U[6] = s.by; U[7] = s.bz;
    F[0] = s.r * s.u;
    F[1] = s.r * s.u * s.u + pT - bn2;
    F[2] = s.r * s.v * s.u - bn * s.by;
    F[3] = s.r * s.w * s.u - bn * s.bz;
    F[4] = (E + pT) * s.u - bn * vb;
    F[5] = T(0);
    F[6] = s.by * s.u - bn * s.v;
    F[7] = s.bz * s.u - bn * s.w;
  };

  T FL[8], UL[8];
  if (SL > T(0)) {
    phys(L, EL, pTL, FL, UL);
    for (int k = 0; k < 8; ++k) out[k] = FL[k];
    set_state(L.u, L.v, L.w, L.by, L.bz);
    return;
  }
  T FR[8], UR[8];
  if (SR < T(0)) {  // the whole fan moves left of the face: the right state's flux
    phys(R, ER, pTR, FR, UR);
    for (int k = 0; k < 8; ++k) out[k] = FR[k];
    set_state(R.u, R.v, R.w, R.by, R.bz);
    return;
  }
  phys(L, EL, pTL, FL, UL);
  phys(R, ER, pTR, FR, UR);
  const T dL = SL - L.u, dR = SR - R.u;
  const T iden = rcp(dR * R.r - dL * L.r);
  const T SM = (dR * R.r * R.u - dL * L.r * L.u - pTR + pTL) * iden;
  const T pTs = (dR * R.r * pTL - dL * L.r * pTR + L.r * R.r * dR * dL * (R.u - L.u)) * iden;

  // single-starred states (Miyoshi & Kusano 2005), side by side without
  // run-time indexing so that everything stays in registers
  const T islm = rcp(SL - SM), isrm = rcp(SR - SM);
  const T rsL = L.r * dL * islm, rsR = R.r * dR * isrm;
  T vsL, wsL, bysL, bzsL, vsR, wsR, bysR, bzsR;
  {
    const T q = L.r * dL * (SL - SM), dd = q - bn2;
    const T aq = q < T(0) ? -q : q, add = dd < T(0) ? -dd : dd;
    if (add < eps * (aq + bn2)) {
      vsL = L.v; wsL = L.w; bysL = L.by; bzsL = L.bz;
    } else {
      const T idd = rcp(dd);
      const T fv = bn * (SM - L.u) * idd, fb = (L.r * dL * dL - bn2) * idd;
      vsL = L.v - L.by * fv; wsL = L.w - L.bz * fv; bysL = L.by * fb; bzsL = L.bz * fb;
    }
  }
  {
    const T q = R.r * dR * (SR - SM), dd = q - bn2;
    const T aq = q < T(0) ? -q : q, add = dd < T(0) ? -dd : dd;
    if (add < eps * (aq + bn2)) {
      vsR = R.v; wsR = R.w; bysR = R.by; bzsR = R.bz;
    } else {
      const T idd = rcp(dd);
      const T fv = bn * (SM - R.u) * idd, fb = (R.r * dR * dR - bn2) * idd;
      vsR = R.v - R.by * fv; wsR = R.w - R.bz * fv; bysR = R.by * fb; bzsR = R.bz * fb;
    }
  }
  const T vbL = L.u * bn + L.v * L.by + L.w * L.bz, vbR = R.u * bn + R.v * R.by + R.w * R.bz;
  const T vbsL = SM * bn + vsL * bysL + wsL * bzsL, vbsR = SM * bn + vsR * bysR + wsR * bzsR;
  const T EsL = (dL * EL - pTL * L.u + pTs * SM + bn * (vbL - vbsL)) * islm;
  const T EsR = (dR * ER - pTR * R.u + pTs * SM + bn * (vbR - vbsR)) * isrm;
  const T isqL = rsq(rsL), isqR = rsq(rsR);
  const T sqL = rsL * isqL, sqR = rsR * isqR;
  const T sgn = bn >= T(0) ? T(1) : T(-1);
  const T abn = bn < T(0) ? -bn : bn;
  const T SsL = SM - abn * isqL, SsR = SM + abn * isqR;

  if (SsL >= T(0)) {  // left single-starred region
    const T Us[8] = {rsL, rsL * SM, rsL * vsL, rsL * wsL, EsL, bn, bysL, bzsL};
    for (int k = 0; k < 8; ++k) out[k] = FL[k] + SL * (Us[k] - UL[k]);
    set_state(SM, vsL, wsL, bysL, bzsL);
    return;
  }
  if (SM < T(0) && SsR < T(0)) {
    if (SR >= T(0)) {  // right single-starred region
      const T Us[8] = {rsR, rsR * SM, rsR * vsR, rsR * wsR, EsR, bn, bysR, bzsR};
      for (int k = 0; k < 8; ++k) out[k] = FR[k] + SR * (Us[k] - UR[k]);
      set_state(SM, vsR, wsR, bysR, bzsR);
    } else {
      for (int k = 0; k < 8; ++k) out[k] = FR[k];
      set_state(R.u, R.v, R.w, R.by, R.bz);
    }
    return;
  }
  // double-starred states
  const T inv = rcp(sqL + sqR);
  const T vss = (sqL * vsL + sqR * vsR + (bysR - bysL) * sgn) * inv;
  const T wss = (sqL * wsL + sqR * wsR + (bzsR - bzsL) * sgn) * inv;
  const T byss = (sqL * bysR + sqR * bysL + sqL * sqR * (vsR - vsL) * sgn) * inv;
  const T bzss = (sqL * bzsR + sqR * bzsL + sqL * sqR * (wsR - wsL) * sgn) * inv;
  const T vbss = SM * bn + vss * byss + wss * bzss;
  set_state(SM, vss, wss, byss, bzss);
  if (SM >= T(0)) {
    const T Ess = EsL - sqL * (vbsL - vbss) * sgn;
    const T Us[8] = {rsL, rsL * SM, rsL * vsL, rsL * wsL, EsL, bn, bysL, bzsL};
    const T Uss[8] = {rsL, rsL * SM, rsL * vss, rsL * wss, Ess, bn, byss, bzss};
    for (int k = 0; k < 8; ++k) out[k] = FL[k] + SL * (Us[k] - UL[k]) + SsL * (Uss[k] - Us[k]);
  } else {
    const T Ess = EsR + sqR * (vbsR - vbss) * sgn;
    const T Us[8] = {rsR, rsR * SM, rsR * vsR, rsR * wsR, EsR, bn, bysR, bzsR};
    const T Uss[8] = {rsR, rsR * SM, rsR * vss, rsR * wss, Ess, bn, byss, bzss};
    for (int k = 0; k < 8; ++k) out[k] = FR[k] + SR * (Us[k] - UR[k]) + SsR * (Uss[k] - Us[k]);
  }
}

// Face flux for a face normal to `a` from conserved traces uL, uR (xyz frame).
// Writes F[0..V-1] in the xyz frame and returns B^n_F. qd (nullable, Powell):
// q^dagger of eq. powellq-interp against the HLLD interface state u_F for the
// left trace (qd[0..6]) and the right trace (qd[7..13]); per side the
// components act on the momentum (B_L + B_F)/2 [0..2], the energy
// (2 B_L.v_L + B_L.v_F + B_F.v_L + 2 B_F.v_F)/6 [3] and the induction
// (v_L + v_F)/2 [4..6] equations, in the xyz frame.
template <typename T>
__device__ __forceinline__ T face_flux(const T* uL, const T* uR, int a, T gamma, bool glm, T ch, T eps,
                                       T* F, T* qd = nullptr) {
  const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
  Prim<T> L, R;
  {
    const T ir = rcp(uL[0]);
    const T v0 = uL[1] * ir, v1 = uL[2] * ir, v2 = uL[3] * ir;
    const T b2 = uL[5] * uL[5] + uL[6] * uL[6] + uL[7] * uL[7];
    L.r = uL[0];
    L.p = (gamma - T(1)) * (uL[4] - T(0.5) * uL[0] * (v0 * v0 + v1 * v1 + v2 * v2) - T(0.5) * b2);
    const T vv[3] = {v0, v1, v2};
    L.u = vv[a]; L.v = vv[t1]; L.w = vv[t2];
    L.by = uL[5 + t1]; L.bz = uL[5 + t2];
  }
  {
    const T ir = rcp(uR[0]);
    const T v0 = uR[1] * ir, v1 = uR[2] * ir, v2 = uR[3] * ir;
    const T b2 = uR[5] * uR[5] + uR[6] * uR[6] + uR[7] * uR[7];
    R.r = uR[0];
    R.p = (gamma - T(1)) * (uR[4] - T(0.5) * uR[0] * (v0 * v0 + v1 * v1 + v2 * v2) - T(0.5) * b2);
    const T vv[3] = {v0, v1, v2};
    R.u = vv[a]; R.v = vv[t1]; R.w = vv[t2];
    R.by = uR[5 + t1]; R.bz = uR[5 + t2];
  }
  const T bnL = uL[5 + a], bnR = uR[5 + a];
  const T bnF = bn_face(L.r, R.r, bnL, bnR);
  T Fr[8];
  Prim<T> sf;
  hlld(L, R, bnF, gamma, eps, Fr, qd ? &sf : nullptr);
  if (qd) {
    T vF[3], BF[3];
    vF[a] = sf.u; vF[t1] = sf.v; vF[t2] = sf.w;
    BF[a] = bnF; BF[t1] = sf.by; BF[t2] = sf.bz;
    for (int side = 0; side < 2; ++side) {
      const T* u = side ? uR : uL;
      const T ir = rcp(u[0]);
      const T vX[3] = {u[1] * ir, u[2] * ir, u[3] * ir};
      const T BX[3] = {u[5], u[6], u[7]};
      T* q = qd + 7 * side;
      T bxvx = T(0), bxvf = T(0), bfvx = T(0), bfvf = T(0);
      for (int k = 0; k < 3; ++k) {
        q[k] = T(0.5) * (BX[k] + BF[k]);
        q[4 + k] = T(0.5) * (vX[k] + vF[k]);
        bxvx += BX[k] * vX[k];
        bxvf += BX[k] * vF[k];
        bfvx += BF[k] * vX[k];
        bfvf += BF[k] * vF[k];
      }
      q[3] = (T(2) * bxvx + bxvf + bfvx + T(2) * bfvf) * (T(1) / T(6));
    }
  }
  F[0] = Fr[0];
  F[1 + a] = Fr[1]; F[1 + t1] = Fr[2]; F[1 + t2] = Fr[3];
  F[4] = Fr[4];
  F[5 + a] = Fr[5]; F[5 + t1] = Fr[6]; F[5 + t2] = Fr[7];
  if (glm) {
    const T bstar = T(0.5) * (bnL + bnR) - quot(uR[8] - uL[8], T(2) * ch);
    const T pstar = T(0.5) * (uL[8] + uR[8]) - T(0.5) * ch * (bnR - bnL);
    F[5 + a] = pstar;
    F[8] = ch * ch * bstar;
  }
  return bnF;
}

// LEN-point dot product of two 16-byte aligned arrays (LEN a multiple of 4)
template <typename T, int LEN>
__device__ __forceinline__ T dotp(const T* a, const T* b) {
  T s = T(0);
  if constexpr (sizeof(T) == 4) {
    const float4* A = reinterpret_cast<const float4*>(a);
    const float4* B = reinterpret_cast<const float4*>(b);
#pragma unroll
    for (int k = 0; k < LEN / 4; ++k) {
      const float4 x = A[k], y = B[k];
      s = fmaf(x.x, y.x, s);
      s = fmaf(x.y, y.y, s);
      s = fmaf(x.z, y.z, s);
      s = fmaf(x.w, y.w, s);
    }
  } else {
    const double2* A = reinterpret_cast<const double2*>(a);
    const double2* B = reinterpret_cast<const double2*>(b);
#pragma unroll
    for (int k = 0; k < LEN / 2; ++k) {
      const double2 x = A[k], y = B[k];
      s = fma(x.x, y.x, s);
      s = fma(x.y, y.y, s);
    }
  }
  return s;
}

}  // namespace dgmhd
