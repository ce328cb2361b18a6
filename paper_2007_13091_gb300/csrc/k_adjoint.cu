// Adjoint of the wave part of the step with the particle part frozen (first
// order; Sec. 2.1, 2.3, 2.4 (d), (e)).
//
// Frozen map: with the recorded time steps dt^n, particle densities rho^p_n
// (rho^h = rho - rho^p) and particle fluxes pf^n of K real steps,
//   W^{n+1}_i = W^n_i - sum_f (+/-) F_f(W^n; theta) |S_f| / |Omega_i| + pf^n_i / |Omega_i|,
// and a wall functional J = sum_n sum_{listed boundary faces} F_f[c] |S_f|
// (c = 1: x momentum delivered to the walls, drag; c = 4: energy, wall heat
// flux).  theta = (rho_inf, U_inf, T_w) parameterises every far-field state
// equal to the first one (density, speed along its direction, its own
// temperature) and the temperature of the listed diffuse walls.
//
// Reverse sweep (hand-written adjoint): lambda^K = 0 and for n = K-1..0
//   g_f      = -|S_f|/|Omega_o| lambda^{n+1}_o + |S_f|/|Omega_nb| lambda^{n+1}_nb
//              + |S_f| e_c  (listed boundary faces),
//   lambda^n = lambda^{n+1} + sum_f (dF_f/dW^n)^T g_f,
//   dJ/dtheta += sum_f (dF_f/dtheta)^T g_f.
// Face states are recomputed from the checkpointed W^n; each face's local
// vector-Jacobian products come from evaluating its flux on dual numbers
// seeded on the owner's W, the neighbour's W and theta in turn.  Per-face
// products are gathered per cell in the fixed order of the cell's faces.
#include "dual.cuh"
#include "ugkwp_internal.hpp"

namespace ugkwp {

namespace {

using ad::Dual;
constexpr double PI = 3.14159265358979323846;

// generic elementary functions: binary64 or dual
__device__ __forceinline__ double sqrt_(double x) { return ::sqrt(x); }
__device__ __forceinline__ double exp_(double x) { return ::exp(x); }
__device__ __forceinline__ double log_(double x) { return ::log(x); }
__device__ __forceinline__ double expm1_(double x) { return ::expm1(x); }
__device__ __forceinline__ double erfc_(double x) { return ::erfc(x); }
__device__ __forceinline__ double fabs_(double x) { return ::fabs(x); }
template <int N> __device__ __forceinline__ Dual<N> sqrt_(const Dual<N>& x) { return ad::sqrt(x); }
template <int N> __device__ __forceinline__ Dual<N> exp_(const Dual<N>& x) { return ad::exp(x); }
template <int N> __device__ __forceinline__ Dual<N> log_(const Dual<N>& x) { return ad::log(x); }
template <int N> __device__ __forceinline__ Dual<N> expm1_(const Dual<N>& x) { return ad::expm1(x); }
template <int N> __device__ __forceinline__ Dual<N> erfc_(const Dual<N>& x) { return ad::erfc(x); }
template <int N> __device__ __forceinline__ Dual<N> fabs_(const Dual<N>& x) { return ad::fabs(x); }

template <class S> struct Prim { S rho, U[3], p, T, lam; };

template <class S> __device__ Prim<S> prim_of(const S* W, double R) {
    Prim<S> s;
    s.rho = W[0];
    const S ir = 1.0 / W[0];
    for (int d = 0; d < 3; ++d) s.U[d] = W[1 + d] * ir;
    const S U2 = s.U[0] * s.U[0] + s.U[1] * s.U[1] + s.U[2] * s.U[2];
    s.p = (W[4] - 0.5 * (s.rho * U2)) * (2.0 / 3.0);
    s.T = s.p / (s.rho * R);
    s.lam = s.rho / (2.0 * s.p);
    return s;
}

// mu(T)/p with mu = mu_ref (T/T_ref)^omega
template <class S> __device__ S tau_of(const S& T, const S& p, const DevParams& P) {
    return P.mu_ref * exp_(P.omega * log_(T * (1.0 / P.T_ref))) / p;
}

// q1, q4 and a4 = q4 - dt e^{-dt/tau}
template <class S> __device__ void coeffs(double dt, const S& tau, S& q1, S& q4, S& a4) {
    const S x = dt / tau;
    if (ad::val(x) < 1.0) {
        S s1 = 0.0, s4 = 0.0, sa = 0.0, term = 1.0;
        for (int k = 1; k <= 30; ++k) {
            term = term * x * (1.0 / (double)k);
            const double sg = (k & 1) ? -1.0 : 1.0;
            if (k >= 2) s1 = s1 + sg * term;
            s4 = s4 - sg * term;
            if (k >= 2) sa = sa + (sg * (double)(k - 1)) * term;
        }
        q1 = tau * s1;
        q4 = tau * s4;
        a4 = tau * sa;
    } else {
        const S em1 = expm1_(-x);
        q4 = -(tau * em1);
        q1 = dt - q4;
        a4 = q4 - dt * (em1 + 1.0);
    }
}

// unit-density half-space (half = +1/-1) or full (0) moments <psi>, <u_n psi>
template <class S> __device__ void moments(const S& Un, const S* Ut, const double* n, const S& lam, int half, S H[5],
                                           S G[5]) {
    S M[5];
    if (half == 0) {
        M[0] = 1.0;
        M[1] = Un;
    } else {
        const S a = sqrt_(lam) * Un;
        const S edge = 0.5 * exp_(-(lam * Un * Un)) / sqrt_(PI * lam);
        if (half > 0) { M[0] = 0.5 * erfc_(-a); M[1] = Un * M[0] + edge; }
        else          { M[0] = 0.5 * erfc_(a);  M[1] = Un * M[0] - edge; }
    }
    const S h = 0.5 / lam;
    for (int k = 0; k < 3; ++k) M[k + 2] = Un * M[k + 1] + (double)(k + 1) * h * M[k];
    const S tv = Ut[0] * Ut[0] + Ut[1] * Ut[1] + Ut[2] * Ut[2] + 2.0 * h;
    H[0] = M[0];
    G[0] = M[1];
    for (int d = 0; d < 3; ++d) {
        H[1 + d] = M[1] * n[d] + M[0] * Ut[d];
        G[1 + d] = M[2] * n[d] + M[1] * Ut[d];
    }
    H[4] = 0.5 * (M[2] + M[0] * tv);
    G[4] = 0.5 * (M[3] + M[1] * tv);
}

template <class S> struct Side { S rho, rhoh, Un, Ut[3], lam, p, T; };

template <class S> __device__ Side<S> side_of(const S* W, const S& rhoh, const double* n, double R) {
    const Prim<S> s = prim_of(W, R);
    Side<S> f;
    f.rho = s.rho; f.rhoh = rhoh; f.lam = s.lam; f.p = s.p; f.T = s.T;
    f.Un = s.U[0] * n[0] + s.U[1] * n[1] + s.U[2] * n[2];
    for (int d = 0; d < 3; ++d) f.Ut[d] = s.U[d] - f.Un * n[d];
    return f;
}

// F = q1 <u_n psi>_{g0} + a4 (upwind hydrodynamic halves); a ghost that
// emits no particles carries q4 on its incoming half
template <class S> __device__ void interior(const Side<S>& L, const Side<S>& R, bool ghost, const double* n, double dt,
                                            const DevParams& P, S F[5]) {
    S HL[5], GL[5], HR[5], GR[5];
    moments(L.Un, L.Ut, n, L.lam, +1, HL, GL);
    moments(R.Un, R.Ut, n, R.lam, -1, HR, GR);
    S W0[5];
    for (int q = 0; q < 5; ++q) W0[q] = L.rho * HL[q] + R.rho * HR[q];
    const Prim<S> s0 = prim_of(W0, P.R);
    S tau = tau_of(s0.T, s0.p, P);
    if (P.C2 > 0.0) tau = tau + P.C2 * fabs_(L.p - R.p) / fabs_(L.p + R.p) * dt;
    S q1, q4, a4;
    coeffs(dt, tau, q1, q4, a4);
    const S Un0 = s0.U[0] * n[0] + s0.U[1] * n[1] + s0.U[2] * n[2];
    S Ut0[3];
    for (int d = 0; d < 3; ++d) Ut0[d] = s0.U[d] - Un0 * n[d];
    S H0[5], G0[5];
    moments(Un0, Ut0, n, s0.lam, 0, H0, G0);
    const S cR = ghost ? q4 : a4;
    for (int k = 0; k < 5; ++k) F[k] = q1 * (s0.rho * G0[k]) + a4 * (L.rhoh * GL[k]) + cR * (R.rhoh * GR[k]);
}

// Flux of face f from the owner's W (and the neighbour's, or the boundary
// condition parameterised by theta).
template <class S> __device__ void face_flux(const DevMesh& m, const DevParams& P, const AdjParams& ap, int f,
                                             const S* WL, double rpL, const S* WR, double rpR, const S* th, double dt,
                                             S F[5]) {
    const int nf = m.nf;
    const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
    const S rhohL = WL[0] - rpL;
    const Side<S> L = side_of(WL, rhohL, n, P.R);
    const int nb = m.f_nbr[f];
    if (nb >= 0) {
        const S rhohR = WR[0] - rpR;
        const Side<S> R = side_of(WR, rhohR, n, P.R);
        interior(L, R, false, n, dt, P, F);
        return;
    }
    const int tag = m.bf_tag[-1 - nb];
    const DevBc& bc = P.bc[tag];
    const AdjBc& ab = ap.b[tag];
    if (bc.type == UGKWP_BC_DIFFUSE_WALL) {
        const S tauL = tau_of(L.T, L.p, P);
        S q1, q4, a4;
        coeffs(dt, tauL, q1, q4, a4);
        S HL[5], GL[5];
        moments(L.Un, L.Ut, n, L.lam, +1, HL, GL);
        S Gin[5];
        for (int k = 0; k < 5; ++k) Gin[k] = q1 * (L.rho * GL[k]) + a4 * (L.rhoh * GL[k]);
        const S Tw = ab.param_wall ? th[2] : S(bc.T_w);
        const S lamw = 1.0 / (2.0 * P.R * Tw);
        const double Uwn = bc.U_w[0] * n[0] + bc.U_w[1] * n[1] + bc.U_w[2] * n[2];
        S Uwt[3];
        for (int d = 0; d < 3; ++d) Uwt[d] = bc.U_w[d] - Uwn * n[d];
        S Hw[5], Gw[5];
        moments(S(Uwn), Uwt, n, lamw, -1, Hw, Gw);
        const S rhow = -Gin[0] / (dt * Gw[0]);
        for (int k = 0; k < 5; ++k) F[k] = Gin[k] + dt * rhow * Gw[k];
        return;
    }
    if (bc.type == UGKWP_BC_SPECULAR) {
        Side<S> R = L;
        R.Un = -L.Un;
        S Ff[5];
        interior(L, R, false, n, dt, P, Ff);
        const S fn = Ff[1] * n[0] + Ff[2] * n[1] + Ff[3] * n[2];
        F[0] = 0.0;
        F[4] = 0.0;
        for (int d = 0; d < 3; ++d) F[1 + d] = fn * n[d];
        return;
    }
    Side<S> R = L;
    if (bc.type == UGKWP_BC_FARFIELD) {
        S Win[5];
        if (ab.param_ff) {
            Win[0] = th[0];
            for (int d = 0; d < 3; ++d) Win[1 + d] = th[0] * th[1] * ab.e[d];
            Win[4] = th[0] * (0.5 * th[1] * th[1] + 1.5 * ab.RT);
        } else {
            for (int q = 0; q < 5; ++q) Win[q] = bc.W_in[q];
        }
        R = side_of(Win, Win[0], n, P.R);
    }
    R.rhoh = R.rho;
    interior(L, R, true, n, dt, P, F);
}

// ---- second order, generic (Sec. 2.1, 2.3): interior faces of a step whose
// limited least-squares gradients are given (their limiter values frozen),
// in the closed forms of the second-order kernel, on binary64 or duals.
template <class S> struct TabS { S n[7], v[7], w[7]; };

template <class S> __device__ void gauss_mom_s(const S& mean, const S& h, S* M) {
    M[0] = S(1.0);
    M[1] = mean;
    for (int k = 0; k < 5; ++k) M[k + 2] = mean * M[k + 1] + ((double)(k + 1) * h) * M[k];
}

template <class S> __device__ void make_tab_s(const S* U, const S& lam, int half, TabS<S>& T) {
    const S h = 0.5 / lam;
    if (half == 0) {
        gauss_mom_s(U[0], h, T.n);
    } else {
        const S a = sqrt_(lam) * U[0];
        const S edge = (0.5 * exp_(-(a * a))) / sqrt_(PI * lam);
        T.n[0] = half > 0 ? 0.5 * erfc_(-a) : 0.5 * erfc_(a);
        T.n[1] = U[0] * T.n[0] + (half > 0 ? edge : -edge);
        for (int k = 0; k < 5; ++k) T.n[k + 2] = U[0] * T.n[k + 1] + ((double)(k + 1) * h) * T.n[k];
    }
    gauss_mom_s(U[1], h, T.v);
    gauss_mom_s(U[2], h, T.w);
}

// <u^AL v^BE w^GA (a.psi) psi_k>, factorised per direction
template <int AL, int BE, int GA, class S> __device__ void apsi_s(const TabS<S>& T, const S* a, S out[5]) {
    const S h4 = 0.5 * a[4];
    S NA[3], VA[3], WA[3];
    for (int i = 0; i < 3; ++i) {
        NA[i] = a[0] * T.n[AL + i] + a[1] * T.n[AL + i + 1] + h4 * T.n[AL + i + 2];
        VA[i] = a[2] * T.v[BE + i + 1] + h4 * T.v[BE + i + 2];
        WA[i] = a[3] * T.w[GA + i + 1] + h4 * T.w[GA + i + 2];
    }
    auto SS = [&](int x, int y, int z) {
        return NA[x] * T.v[BE + y] * T.w[GA + z] + T.n[AL + x] * (VA[y] * T.w[GA + z] + T.v[BE + y] * WA[z]);
    };
    out[0] = SS(0, 0, 0);
    out[1] = SS(1, 0, 0);
    out[2] = SS(0, 1, 0);
    out[3] = SS(0, 0, 1);
    out[4] = 0.5 * (SS(2, 0, 0) + SS(0, 2, 0) + SS(0, 0, 2));
}

template <int AL, class S> __device__ void psi_mom_s(const TabS<S>& T, S out[5]) {
    out[0] = T.n[AL];
    out[1] = T.n[AL + 1];
    out[2] = T.n[AL] * T.v[1];
    out[3] = T.n[AL] * T.w[1];
    out[4] = 0.5 * (T.n[AL + 2] + T.n[AL] * (T.v[2] + T.w[2]));
}

template <class S> __device__ void slope_mom_s(const TabS<S>& T, int d, const S* a, S out[5]) {
    if (d == 0) apsi_s<2, 0, 0>(T, a, out);
    else if (d == 1) apsi_s<1, 1, 0>(T, a, out);
    else apsi_s<1, 0, 1>(T, a, out);
}

// <psi psi^T> a = b for the unit Maxwellian (U, lambda), closed form
template <class S> __device__ void micro_s(const S* U, const S& lam, const S& th, const S* b, S* a) {
    const S R1 = b[1] - U[0] * b[0], R2 = b[2] - U[1] * b[0], R3 = b[3] - U[2] * b[0];
    const S U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const S R4 = 2.0 * b[4] - (U2 + 3.0 * th) * b[0];
    a[4] = (4.0 / 3.0) * lam * lam * (R4 - 2.0 * (U[0] * R1 + U[1] * R2 + U[2] * R3));
    a[1] = 2.0 * lam * R1 - U[0] * a[4];
    a[2] = 2.0 * lam * R2 - U[1] * a[4];
    a[3] = 2.0 * lam * R3 - U[2] * a[4];
    a[0] = b[0] - (U[0] * a[1] + U[1] * a[2] + U[2] * a[3]) - 0.5 * a[4] * (U2 + 3.0 * th);
}

// derivatives of the Maxwellian moments along a conservative slope b
template <class S> struct DPrimS { S dr, dU[3], dth, UdU; };
template <class S> __device__ DPrimS<S> dprim_s(const S* U, const S& th, const S& U2, const S* b) {
    DPrimS<S> q;
    q.dr = b[0];
    for (int j = 0; j < 3; ++j) q.dU[j] = b[1 + j] - U[j] * b[0];
    q.UdU = U[0] * q.dU[0] + U[1] * q.dU[1] + U[2] * q.dU[2];
    q.dth = ((2.0 * b[4] - (U2 + 3.0 * th) * b[0]) - 2.0 * q.UdU) * (1.0 / 3.0);
    return q;
}
template <int D, class S>
__device__ void euler_jac_s(const S* U, const S& th, const S& U2, const S* b, const DPrimS<S>& q, S out[5]) {
    out[0] = b[1 + D];
    for (int j = 0; j < 3; ++j) {
        S v = q.dr * (U[D] * U[j]) + q.dU[D] * U[j] + U[D] * q.dU[j];
        if (j == D) v = v + q.dr * th + q.dth;
        out[1 + j] = v;
    }
    out[4] = b[1 + D] * (0.5 * U2 + 2.5 * th) + U[D] * (q.UdU + 2.5 * q.dth);
}
template <int D, class S> __device__ void q_jac_s(const S* U, const S& th, const S& U2, const DPrimS<S>& q, S out[5]) {
    const S un_ud = U[0] * U[D];
    const S d_un_ud = q.dU[0] * U[D] + U[0] * q.dU[D];
    out[0] = q.dr * un_ud + d_un_ud;
    if (D == 0) out[0] = out[0] + q.dr * th + q.dth;
    for (int j = 0; j < 3; ++j) {
        S sv = S(0.0), ds = S(0.0);
        if (D == j) { sv = sv + U[0]; ds = ds + q.dU[0]; }
        if (j == 0) { sv = sv + U[D]; ds = ds + q.dU[D]; }
        if (D == 0) { sv = sv + U[j]; ds = ds + q.dU[j]; }
        out[1 + j] = q.dr * (un_ud * U[j] + th * sv) + d_un_ud * U[j] + un_ud * q.dU[j] + q.dth * sv + th * ds;
    }
    const S A = U2 + 7.0 * th;
    S v = q.dr * (0.5 * un_ud * A) + 0.5 * (d_un_ud * A + un_ud * (2.0 * q.UdU + 7.0 * q.dth));
    if (D == 0) {
        const S Bq = U2 + 5.0 * th;
        v = v + q.dr * (0.5 * th * Bq) + 0.5 * (q.dth * Bq + th * (2.0 * q.UdU + 5.0 * q.dth));
    }
    out[4] = v;
}

template <class S> struct QCS { S q1, q2, q3, q4, q5, a4, a5; };
template <class S> __device__ QCS<S> time_coeffs_s(double dt, const S& tau) {
    QCS<S> c;
    const S em1 = expm1_(-(dt / tau));
    const S e = 1.0 + em1;
    const S tdt = tau * dt;
    c.q4 = -(tau * em1);
    c.q1 = dt - c.q4;
    c.a4 = c.q4 - dt * e;
    c.q2 = 2.0 * tau * c.q4 - tdt - tdt * e;
    c.q3 = 0.5 * dt * dt - tdt + tau * c.q4;
    c.q5 = tdt * e - tau * c.q4;
    c.a5 = c.q5 + 0.5 * dt * dt * e;
    return c;
}

__device__ void face_frame_d(const double* n, double R[3][3]) {
    int ax = 0;
    if (::fabs(n[1]) < ::fabs(n[ax])) ax = 1;
    if (::fabs(n[2]) < ::fabs(n[ax])) ax = 2;
    double t1[3];
    t1[0] = ax == 0 ? 0.0 : (ax == 1 ? n[2] : -n[1]);
    t1[1] = ax == 1 ? 0.0 : (ax == 0 ? -n[2] : n[0]);
    t1[2] = ax == 2 ? 0.0 : (ax == 0 ? n[1] : -n[0]);
    const double il = rsqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int d = 0; d < 3; ++d) t1[d] *= il;
    R[0][0] = n[0]; R[0][1] = n[1]; R[0][2] = n[2];
    R[1][0] = t1[0]; R[1][1] = t1[1]; R[1][2] = t1[2];
    R[2][0] = n[1] * t1[2] - n[2] * t1[1];
    R[2][1] = n[2] * t1[0] - n[0] * t1[2];
    R[2][2] = n[0] * t1[1] - n[1] * t1[0];
}

template <class S> struct SideS { S rho, rhoh, p, H[5], G[5], S5[5]; };

// One side at second order in the face frame: W, rho^h and their lab
// gradients gW [3q + d], gH [d] reconstructed at the face (first order if the
// reconstruction is not positive); B accumulates half of the frame slopes.
template <class S>
__device__ SideS<S> side_o2_s(const S* Wc, const S& rhohc, const S* gW, const S* gH, const double* dx,
                              const double R[3][3], int half, S B[3][5], bool first) {
    S Wf[5];
    for (int q = 0; q < 5; ++q) Wf[q] = Wc[q] + gW[3 * q] * dx[0] + gW[3 * q + 1] * dx[1] + gW[3 * q + 2] * dx[2];
    S rh = rhohc + gH[0] * dx[0] + gH[1] * dx[1] + gH[2] * dx[2];
    S pr = (Wf[4] - 0.5 * (Wf[1] * Wf[1] + Wf[2] * Wf[2] + Wf[3] * Wf[3]) / Wf[0]) * (2.0 / 3.0);
    const bool o2 = ad::val(Wf[0]) > 0.0 && ad::val(pr) > 0.0;
    if (!o2) {
        for (int q = 0; q < 5; ++q) Wf[q] = Wc[q];
        rh = rhohc;
        pr = (Wf[4] - 0.5 * (Wf[1] * Wf[1] + Wf[2] * Wf[2] + Wf[3] * Wf[3]) / Wf[0]) * (2.0 / 3.0);
    }
    SideS<S> o;
    S W[5];
    W[0] = Wf[0];
    for (int j = 0; j < 3; ++j) W[1 + j] = R[j][0] * Wf[1] + R[j][1] * Wf[2] + R[j][2] * Wf[3];
    W[4] = Wf[4];
    o.rho = W[0];
    o.rhoh = rh;
    o.p = pr;
    const S ir = 1.0 / W[0];
    const S U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const S lam = 0.5 * W[0] / pr;
    const S th = 0.5 / lam;
    TabS<S> T;
    make_tab_s(U, lam, half, T);
    psi_mom_s<0>(T, o.H);
    psi_mom_s<1>(T, o.G);
    for (int k = 0; k < 5; ++k) o.S5[k] = S(0.0);
    if (!o2) {
        if (first)
            for (int dd = 0; dd < 3; ++dd)
                for (int q = 0; q < 5; ++q) B[dd][q] = S(0.0);
        return o;
    }
    const S ratio = rh * ir;
    for (int dd = 0; dd < 3; ++dd) {
        S g[5], dW[5], b[5], a[5], sm[5];
        for (int q = 0; q < 5; ++q) g[q] = gW[3 * q] * R[dd][0] + gW[3 * q + 1] * R[dd][1] + gW[3 * q + 2] * R[dd][2];
        dW[0] = g[0];
        for (int j = 0; j < 3; ++j) dW[1 + j] = R[j][0] * g[1] + R[j][1] * g[2] + R[j][2] * g[3];
        dW[4] = g[4];
        for (int q = 0; q < 5; ++q) B[dd][q] = first ? 0.5 * dW[q] : B[dd][q] + 0.5 * dW[q];
        const S gh = gH[0] * R[dd][0] + gH[1] * R[dd][1] + gH[2] * R[dd][2];
        const S gr = (gh - ratio * dW[0]) * ir;
        for (int q = 0; q < 5; ++q) b[q] = ratio * dW[q] + W[q] * gr;
        micro_s(U, lam, th, b, a);
        slope_mom_s(T, dd, a, sm);
        for (int k = 0; k < 5; ++k) o.S5[k] = o.S5[k] + sm[k];
    }
    return o;
}

// Second-order flux of an interior face (lab frame, per unit area).
template <class S>
__device__ void interior_o2_s(const S* WL, const S& rhL, const S* gWL, const S* gHL, const double* dxL, const S* WR,
                              const S& rhR, const S* gWR, const S* gHR, const double* dxR, const double* n, double dt,
                              const DevParams& P, S F[5]) {
    double R[3][3];
    face_frame_d(n, R);
    S B[3][5];
    const SideS<S> L = side_o2_s(WL, rhL, gWL, gHL, dxL, R, +1, B, true);
    const SideS<S> Rs = side_o2_s(WR, rhR, gWR, gHR, dxR, R, -1, B, false);
    S W0[5];
    for (int k = 0; k < 5; ++k) W0[k] = L.rho * L.H[k] + Rs.rho * Rs.H[k];
    const S rho0 = W0[0], ir0 = 1.0 / rho0;
    const S U0[3] = {W0[1] * ir0, W0[2] * ir0, W0[3] * ir0};
    const S U20 = U0[0] * U0[0] + U0[1] * U0[1] + U0[2] * U0[2];
    const S p0 = (W0[4] - 0.5 * rho0 * U20) * (2.0 / 3.0);
    const S T0 = p0 * ir0 / P.R;
    S tau = tau_of(T0, p0, P);
    if (P.C2 > 0.0) tau = tau + P.C2 * fabs_(L.p - Rs.p) / fabs_(L.p + Rs.p) * dt;
    const QCS<S> qc = time_coeffs_s(dt, tau);
    for (int k = 0; k < 5; ++k) F[k] = qc.a4 * (L.rhoh * L.G[k] + Rs.rhoh * Rs.G[k]) + qc.a5 * (L.S5[k] + Rs.S5[k]);
    const S th0 = p0 * ir0;
    S Fe[5];
    Fe[0] = qc.q1 * W0[1];
    for (int j = 0; j < 3; ++j) Fe[1 + j] = qc.q1 * (W0[1] * U0[j]) + (j == 0 ? qc.q1 * p0 : S(0.0));
    Fe[4] = qc.q1 * U0[0] * (W0[4] + p0);
    S Wt[5], t5[5];
    {
        const DPrimS<S> q = dprim_s(U0, th0, U20, B[0]);
        q_jac_s<0>(U0, th0, U20, q, t5);
        for (int k = 0; k < 5; ++k) Fe[k] = Fe[k] + qc.q2 * t5[k];
        euler_jac_s<0>(U0, th0, U20, B[0], q, t5);
        for (int k = 0; k < 5; ++k) Wt[k] = -t5[k];
    }
    {
        const DPrimS<S> q = dprim_s(U0, th0, U20, B[1]);
        q_jac_s<1>(U0, th0, U20, q, t5);
        for (int k = 0; k < 5; ++k) Fe[k] = Fe[k] + qc.q2 * t5[k];
        euler_jac_s<1>(U0, th0, U20, B[1], q, t5);
        for (int k = 0; k < 5; ++k) Wt[k] = Wt[k] - t5[k];
    }
    {
        const DPrimS<S> q = dprim_s(U0, th0, U20, B[2]);
        q_jac_s<2>(U0, th0, U20, q, t5);
        for (int k = 0; k < 5; ++k) Fe[k] = Fe[k] + qc.q2 * t5[k];
        euler_jac_s<2>(U0, th0, U20, B[2], q, t5);
        for (int k = 0; k < 5; ++k) Wt[k] = Wt[k] - t5[k];
    }
    {
        const DPrimS<S> q = dprim_s(U0, th0, U20, Wt);
        euler_jac_s<0>(U0, th0, U20, Wt, q, t5);
        for (int k = 0; k < 5; ++k) Fe[k] = Fe[k] + qc.q3 * t5[k];
    }
    if (P.pr_fix != 0.0) {
        S mo[5];
        for (int k = 0; k < 5; ++k) mo[k] = qc.q1 * W0[k] + (qc.q3 - qc.q2) * Wt[k];
        const S qf = (Fe[4] - ((U0[0] * Fe[1] + U0[1] * Fe[2]) + U0[2] * Fe[3])) + 0.5 * U20 * Fe[0];
        const S qm = (mo[4] - ((U0[0] * mo[1] + U0[1] * mo[2]) + U0[2] * mo[3])) + 0.5 * U20 * mo[0];
        Fe[4] = Fe[4] + P.pr_fix * (qf - U0[0] * qm);
    }
    for (int k = 0; k < 5; ++k) F[k] = F[k] + Fe[k];
    const S Fm[3] = {F[1], F[2], F[3]};
    for (int d = 0; d < 3; ++d) F[1 + d] = Fm[0] * R[0][d] + Fm[1] * R[1][d] + Fm[2] * R[2][d];
}

__device__ __forceinline__ bool listed_face(const DevMesh& m, const AdjParams& ap, int f) {
    const int nb = m.f_nbr[f];
    return nb < 0 && ap.b[m.bf_tag[-1 - nb]].listed;
}

// far-field state of tag b at theta (or as given)
__device__ __forceinline__ void farfield_state(const DevParams& P, const AdjParams& ap, int tag, const double* th,
                                               double* Win) {
    const DevBc& bc = P.bc[tag];
    const AdjBc& ab = ap.b[tag];
    if (ab.param_ff) {
        Win[0] = th[0];
        for (int d = 0; d < 3; ++d) Win[1 + d] = th[0] * th[1] * ab.e[d];
        Win[4] = th[0] * (0.5 * th[1] * th[1] + 1.5 * ab.RT);
    } else {
        for (int q = 0; q < 5; ++q) Win[q] = bc.W_in[q];
    }
}

// Limited least-squares gradients of W and rho^h = rho - rho^p (second order):
// one thread per (quantity, cell), as in the step; with record the limiter
// values are computed and stored in phi [6][nc], otherwise phi is used as
// given (the limiter frozen at theta).  Far-field ghosts hold the state at theta.
__global__ void __launch_bounds__(128) k_adj_grad(DevMesh m, DevParams P, AdjParams ap, const double* W,
                                                  const double* rho_p, const double* theta, double* phi, int record,
                                                  double* gW, double* gH) {
    const int nc = m.nc;
    const double th[3] = {theta[0], theta[1], theta[2]};
    const long long n = 6LL * nc;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / nc);
        const int i = (int)(t - (long long)q * nc);
        const int own = m.cfs[i];
        const double self = q < 5 ? W[(size_t)q * nc + i] : W[i] - rho_p[i];
        double val[4];
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            const int other = ((own >> k) & 1) ? m.f_nbr[f] : m.f_own[f];
            if (other >= 0) {
                val[k] = q < 5 ? W[(size_t)q * nc + other] : W[other] - rho_p[other];
            } else {
                const int b = -1 - other;
                const int tag = m.bf_tag[b];
                const DevBc& bc = P.bc[tag];
                val[k] = self;
                if (bc.type == UGKWP_BC_SPECULAR && q >= 1 && q <= 3) {
                    const int nbf = m.nbf;
                    double nn[3];
                    for (int d = 0; d < 3; ++d) nn[d] = m.bf_n[(size_t)d * nbf + b];
                    const double mn = W[(size_t)nc + i] * nn[0] + W[(size_t)2 * nc + i] * nn[1] + W[(size_t)3 * nc + i] * nn[2];
                    val[k] = self - 2.0 * mn * nn[q - 1];
                } else if (bc.type == UGKWP_BC_FARFIELD) {
                    double Win[5];
                    farfield_state(P, ap, tag, th, Win);
                    val[k] = q < 5 ? Win[q] : Win[0];
                }
            }
        }
        double g[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) g[d] += m.lsq_c[(size_t)(3 * k + d) * nc + i] * (val[k] - self);
        double ph;
        if (record) {
            double vmax = self, vmin = self;
            for (int k = 0; k < 4; ++k) { vmax = fmax(vmax, val[k]); vmin = fmin(vmin, val[k]); }
            const double eps2 = m.eps2[i];
            double bn = 1.0, bd = 1.0;
            for (int k = 0; k < 4; ++k) {
                const double d2 = g[0] * m.lsq_dxf[(size_t)(3 * k) * nc + i] + g[1] * m.lsq_dxf[(size_t)(3 * k + 1) * nc + i] +
                                  g[2] * m.lsq_dxf[(size_t)(3 * k + 2) * nc + i];
                if (d2 == 0.0) continue;
                const double d1 = d2 > 0.0 ? vmax - self : vmin - self;
                double num = (d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1;
                double den = d2 * (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
                if (den < 0.0) { num = -num; den = -den; }
                if (num * bd < bn * den) { bn = num; bd = den; }
            }
            ph = bn / bd;
            phi[(size_t)q * nc + i] = ph;
        } else {
            ph = phi[(size_t)q * nc + i];
        }
        for (int d = 0; d < 3; ++d) {
            if (q < 5) gW[(size_t)(3 * q + d) * nc + i] = ph * g[d];
            else gH[(size_t)d * nc + i] = ph * g[d];
        }
    }
}

__device__ __forceinline__ void load_grad(const double* gW, const double* gH, int nc, int c, double* gw, double* gh) {
    for (int j = 0; j < 15; ++j) gw[j] = gW[(size_t)j * nc + c];
    for (int d = 0; d < 3; ++d) gh[d] = gH[(size_t)d * nc + c];
}

// the owner's and the neighbour's centroid-to-face vectors of an interior face
__device__ __forceinline__ void face_dx(const DevMesh& m, int f, int o, int nb, double* dxL, double* dxR) {
    const int nc = m.nc;
    const int lk = m.f_lk[f];
    for (int d = 0; d < 3; ++d) {
        dxL[d] = m.lsq_dxf[(size_t)(3 * (lk & 3) + d) * nc + o];
        dxR[d] = m.lsq_dxf[(size_t)(3 * ((lk >> 2) & 3) + d) * nc + nb];
    }
}

// ---- forward: fluxes and the functional's face terms at theta
template <bool O2>
__global__ void __launch_bounds__(128) k_adj_fwd_flux(DevMesh m, DevParams P, AdjParams ap, const double* W,
                                                      const double* rho_p, double dt, const double* theta,
                                                      const double* gW, const double* gH, double* F, double* jf) {
    const int nc = m.nc, nf = m.nf;
    const double th[3] = {theta[0], theta[1], theta[2]};
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const int o = m.f_own[f], nb = m.f_nbr[f];
        double WL[5], WR[5];
        for (int q = 0; q < 5; ++q) {
            WL[q] = W[(size_t)q * nc + o];
            WR[q] = nb >= 0 ? W[(size_t)q * nc + nb] : 0.0;
        }
        double Fv[5];
        if (O2 && nb >= 0) {
            double gwl[15], ghl[3], gwr[15], ghr[3], dxL[3], dxR[3];
            load_grad(gW, gH, nc, o, gwl, ghl);
            load_grad(gW, gH, nc, nb, gwr, ghr);
            face_dx(m, f, o, nb, dxL, dxR);
            const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
            interior_o2_s<double>(WL, WL[0] - rho_p[o], gwl, ghl, dxL, WR, WR[0] - rho_p[nb], gwr, ghr, dxR, n, dt, P, Fv);
        } else {
            face_flux<double>(m, P, ap, f, WL, rho_p[o], WR, nb >= 0 ? rho_p[nb] : 0.0, th, dt, Fv);
        }
        for (int q = 0; q < 5; ++q) F[(size_t)q * nf + f] = Fv[q];
        jf[f] = listed_face(m, ap, f) ? Fv[ap.comp] * m.f_area[f] : 0.0;
    }
}

__global__ void k_adj_update(DevMesh m, const double* W, const double* F, const double* pf, double* Wn) {
    const int nc = m.nc, nf = m.nf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int own = m.cfs[i];
    for (int q = 0; q < 5; ++q) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            const double v = F[(size_t)q * nf + f] * m.f_area[f];
            acc += ((own >> k) & 1) ? v : -v;
        }
        Wn[(size_t)q * nc + i] = (W[(size_t)q * nc + i] - acc / m.vol[i]) + pf[(size_t)q * nc + i] / m.vol[i];
    }
}

// out[c] (+)= sum_j x[c n + j] for c < ncomp (one block, fixed order per thread)
__global__ void k_adj_sum(const double* x, int n, int ncomp, double* out, int accumulate) {
    __shared__ double sh[256];
    for (int c = 0; c < ncomp; ++c) {
        double a = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) a += x[(size_t)c * n + j];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = accumulate ? out[c] + sh[0] : sh[0];
        __syncthreads();
    }
}

// ---- reverse: per face, g_f and its products with the local Jacobians
template <bool O2>
__global__ void __launch_bounds__(128) k_adj_face(DevMesh m, DevParams P, AdjParams ap, const double* W,
                                                  const double* rho_p, double dt, const double* theta,
                                                  const double* gW, const double* gH, const double* lam_next,
                                                  double* wbar, double* gbar, double* thbar) {
    const int nc = m.nc, nf = m.nf;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
        const int o = m.f_own[f], nb = m.f_nbr[f];
        const double area = m.f_area[f];
        double g[5];
        for (int q = 0; q < 5; ++q) {
            g[q] = -area / m.vol[o] * lam_next[(size_t)q * nc + o];
            if (nb >= 0) g[q] += area / m.vol[nb] * lam_next[(size_t)q * nc + nb];
        }
        if (listed_face(m, ap, f)) g[ap.comp] += area;
        const double rpL = rho_p[o], rpR = nb >= 0 ? rho_p[nb] : 0.0;
        if (O2 && nb >= 0) {
            // second order: products with the face's Jacobians with respect to
            // both cells' W and limited gradients, five directions at a time
            double gw[2][15], gh[2][3], dxL[3], dxR[3], Wc[2][5];
            load_grad(gW, gH, nc, o, gw[0], gh[0]);
            load_grad(gW, gH, nc, nb, gw[1], gh[1]);
            face_dx(m, f, o, nb, dxL, dxR);
            for (int q = 0; q < 5; ++q) {
                Wc[0][q] = W[(size_t)q * nc + o];
                Wc[1][q] = W[(size_t)q * nc + nb];
            }
            const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
            // pass: 0/1 W of owner/neighbour, 2..4 / 5..7 gradients of W along
            // x, y, z of owner/neighbour, 8/9 gradient of rho^h of owner/neighbour
            for (int pass = 0; pass < 10; ++pass) {
                Dual<5> WL[5], WR[5], GWL[15], GWR[15], GHL[3], GHR[3], F[5];
                for (int q = 0; q < 5; ++q) {
                    WL[q] = Dual<5>(Wc[0][q]);
                    WR[q] = Dual<5>(Wc[1][q]);
                }
                for (int j = 0; j < 15; ++j) {
                    GWL[j] = Dual<5>(gw[0][j]);
                    GWR[j] = Dual<5>(gw[1][j]);
                }
                for (int d = 0; d < 3; ++d) {
                    GHL[d] = Dual<5>(gh[0][d]);
                    GHR[d] = Dual<5>(gh[1][d]);
                }
                int nseed = 5;
                if (pass == 0) for (int q = 0; q < 5; ++q) WL[q].d[q] = 1.0;
                else if (pass == 1) for (int q = 0; q < 5; ++q) WR[q].d[q] = 1.0;
                else if (pass <= 4) for (int q = 0; q < 5; ++q) GWL[3 * q + (pass - 2)].d[q] = 1.0;
                else if (pass <= 7) for (int q = 0; q < 5; ++q) GWR[3 * q + (pass - 5)].d[q] = 1.0;
                else if (pass == 8) { for (int d = 0; d < 3; ++d) GHL[d].d[d] = 1.0; nseed = 3; }
                else { for (int d = 0; d < 3; ++d) GHR[d].d[d] = 1.0; nseed = 3; }
                interior_o2_s<Dual<5>>(WL, WL[0] - rpL, GWL, GHL, dxL, WR, WR[0] - rpR, GWR, GHR, dxR, n, dt, P, F);
                for (int j = 0; j < nseed; ++j) {
                    double a = 0.0;
                    for (int q = 0; q < 5; ++q) a += g[q] * F[q].d[j];
                    // gbar rows: side s (0 owner, 1 neighbour) x (3q + d for W, 15 + d for rho^h)
                    if (pass == 0) wbar[(size_t)j * nf + f] = a;
                    else if (pass == 1) wbar[(size_t)(5 + j) * nf + f] = a;
                    else if (pass <= 4) gbar[(size_t)(3 * j + (pass - 2)) * nf + f] = a;
                    else if (pass <= 7) gbar[(size_t)(18 + 3 * j + (pass - 5)) * nf + f] = a;
                    else if (pass == 8) gbar[(size_t)(15 + j) * nf + f] = a;
                    else gbar[(size_t)(18 + 15 + j) * nf + f] = a;
                }
            }
            for (int k = 0; k < 3; ++k) thbar[(size_t)k * nf + f] = 0.0;
            continue;
        }
        if (O2)  // a boundary face at second order: first order, no gradient products
            for (int j = 0; j < 36; ++j) gbar[(size_t)j * nf + f] = 0.0;
        // owner's W
        {
            Dual<5> WL[5], WR[5], th[3], F[5];
            for (int q = 0; q < 5; ++q) {
                WL[q] = Dual<5>(W[(size_t)q * nc + o]);
                WL[q].d[q] = 1.0;
                WR[q] = Dual<5>(nb >= 0 ? W[(size_t)q * nc + nb] : 0.0);
            }
            for (int k = 0; k < 3; ++k) th[k] = Dual<5>(theta[k]);
            face_flux<Dual<5>>(m, P, ap, f, WL, rpL, WR, rpR, th, dt, F);
            for (int j = 0; j < 5; ++j) {
                double a = 0.0;
                for (int q = 0; q < 5; ++q) a += g[q] * F[q].d[j];
                wbar[(size_t)j * nf + f] = a;
            }
        }
        if (nb >= 0) {
            Dual<5> WL[5], WR[5], th[3], F[5];
            for (int q = 0; q < 5; ++q) {
                WL[q] = Dual<5>(W[(size_t)q * nc + o]);
                WR[q] = Dual<5>(W[(size_t)q * nc + nb]);
                WR[q].d[q] = 1.0;
            }
            for (int k = 0; k < 3; ++k) th[k] = Dual<5>(theta[k]);
            face_flux<Dual<5>>(m, P, ap, f, WL, rpL, WR, rpR, th, dt, F);
            for (int j = 0; j < 5; ++j) {
                double a = 0.0;
                for (int q = 0; q < 5; ++q) a += g[q] * F[q].d[j];
                wbar[(size_t)(5 + j) * nf + f] = a;
            }
            for (int k = 0; k < 3; ++k) thbar[(size_t)k * nf + f] = 0.0;
        } else {
            for (int j = 0; j < 5; ++j) wbar[(size_t)(5 + j) * nf + f] = 0.0;
            const AdjBc& ab = ap.b[m.bf_tag[-1 - nb]];
            if (ab.param_ff || ab.param_wall) {
                Dual<3> WL[5], WR[5], th[3], F[5];
                for (int q = 0; q < 5; ++q) {
                    WL[q] = Dual<3>(W[(size_t)q * nc + o]);
                    WR[q] = Dual<3>(0.0);
                }
                for (int k = 0; k < 3; ++k) {
                    th[k] = Dual<3>(theta[k]);
                    th[k].d[k] = 1.0;
                }
                face_flux<Dual<3>>(m, P, ap, f, WL, rpL, WR, rpR, th, dt, F);
                for (int k = 0; k < 3; ++k) {
                    double a = 0.0;
                    for (int q = 0; q < 5; ++q) a += g[q] * F[q].d[k];
                    thbar[(size_t)k * nf + f] = a;
                }
            } else {
                for (int k = 0; k < 3; ++k) thbar[(size_t)k * nf + f] = 0.0;
            }
        }
    }
}

// Second order: gg = phi * (sum over the cell's faces of the products with
// its limited gradients) [18][nc], row 3q + d (q = 5: rho^h).
__global__ void k_adj_gg(DevMesh m, const double* phi, const double* gbar, double* gg) {
    const int nc = m.nc, nf = m.nf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int own = m.cfs[i];
    for (int j = 0; j < 18; ++j) {
        double a = 0.0;
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            a += gbar[(size_t)((((own >> k) & 1) ? 0 : 18) + j) * nf + f];
        }
        gg[(size_t)j * nc + i] = phi[(size_t)(j / 3) * nc + i] * a;
    }
}

// lambda^n = lambda^{n+1} + the products of the cell's faces; at second order
// also the gradients' dependence on the cell's W: gradient_c,q = phi sum_k
// c_k (val_k - self_q) is linear in the cell's own value (-c_k), in its
// neighbours' values (+c_k at the neighbour's side) and in the ghost values
// (specular: mirrored momentum; far field: the state at theta, whose theta
// products go to thc [3][nc]).
__global__ void k_adj_cell(DevMesh m, DevParams P, AdjParams ap, const double* W, const double* theta,
                           const double* lam_next, const double* wbar, const double* gg, double* lam, double* thc) {
    const int nc = m.nc, nf = m.nf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int own = m.cfs[i];
    double l[5];
    for (int q = 0; q < 5; ++q) {
        double a = lam_next[(size_t)q * nc + i];
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            a += wbar[(size_t)(((own >> k) & 1) ? q : 5 + q) * nf + f];
        }
        l[q] = a;
    }
    double tc[3] = {0.0, 0.0, 0.0};
    if (P.order == 2) {
        const double th[3] = {theta[0], theta[1], theta[2]};
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            const bool is_own = (own >> k) & 1;
            const int other = is_own ? m.f_nbr[f] : m.f_own[f];
            for (int q = 0; q < 6; ++q) {
                const int dq = q < 5 ? q : 0;  // rho^h = rho - rho^p
                double sself = 0.0;
                for (int d = 0; d < 3; ++d) sself += gg[(size_t)(3 * q + d) * nc + i] * m.lsq_c[(size_t)(3 * k + d) * nc + i];
                if (other >= 0) {
                    const int lk = m.f_lk[f];
                    const int ko = is_own ? ((lk >> 2) & 3) : (lk & 3);
                    double snb = 0.0;
                    for (int d = 0; d < 3; ++d)
                        snb += gg[(size_t)(3 * q + d) * nc + other] * m.lsq_c[(size_t)(3 * ko + d) * nc + other];
                    l[dq] += snb - sself;
                    continue;
                }
                const int b = -1 - other;
                const int tag = m.bf_tag[b];
                const DevBc& bc = P.bc[tag];
                if (bc.type == UGKWP_BC_SPECULAR && q >= 1 && q <= 3) {
                    const int nbf = m.nbf;
                    double nn[3];
                    for (int d = 0; d < 3; ++d) nn[d] = m.bf_n[(size_t)d * nbf + b];
                    for (int jj = 0; jj < 3; ++jj) l[1 + jj] += sself * (-2.0 * nn[q - 1] * nn[jj]);
                } else if (bc.type == UGKWP_BC_FARFIELD) {
                    l[dq] -= sself;
                    const AdjBc& ab = ap.b[tag];
                    if (ab.param_ff) {
                        // d W_in / d theta: rho = th0, m = th0 th1 e, E = th0 (th1^2/2 + 3/2 RT)
                        const int qq = q < 5 ? q : 0;
                        double d0, d1;
                        if (qq == 0) { d0 = 1.0; d1 = 0.0; }
                        else if (qq <= 3) { d0 = th[1] * ab.e[qq - 1]; d1 = th[0] * ab.e[qq - 1]; }
                        else { d0 = 0.5 * th[1] * th[1] + 1.5 * ab.RT; d1 = th[0] * th[1]; }
                        tc[0] += sself * d0;
                        tc[1] += sself * d1;
                    }
                }
            }
        }
    }
    for (int q = 0; q < 5; ++q) lam[(size_t)q * nc + i] = l[q];
    if (thc)
        for (int k = 0; k < 3; ++k) thc[(size_t)k * nc + i] = tc[k];
}

// recorded particle data of the step just taken
__global__ void k_adj_record(DevMesh m, DevState s, DevParams P, double* rho_p, double* pf) {
    const int nc = m.nc;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    rho_p[i] = s.prim[i] - s.rhoh[i];
    for (int q = 0; q < 5; ++q) pf[(size_t)q * nc + i] = (double)s.pflux[(size_t)q * nc + i] * P.qscale[q];
}

}  // namespace

void launch_adj_record(const DevMesh& m, const DevState& s, const DevParams& p, double* rho_p, double* pf,
                       cudaStream_t st) {
    k_adj_record<<<(m.nc + 255) / 256, 256, 0, st>>>(m, s, p, rho_p, pf);
}

static int grad_grid(const DevMesh& m) { return (int)((6LL * m.nc + 127) / 128); }

void launch_adj_forward(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W, const double* rho_p,
                        const double* pf, double dt, const double* theta, const AdjO2& o2, double* F, double* jf,
                        double* Jn, double* Wn, cudaStream_t st) {
    const int g = (m.nf + 127) / 128;
    if (p.order == 2) k_adj_grad<<<grad_grid(m), 128, 0, st>>>(m, p, ap, W, rho_p, theta, o2.phi, 1, o2.gW, o2.gH);
    if (p.order == 2) k_adj_fwd_flux<true><<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, o2.gW, o2.gH, F, jf);
    else k_adj_fwd_flux<false><<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, o2.gW, o2.gH, F, jf);
    k_adj_sum<<<1, 256, 0, st>>>(jf, m.nf, 1, Jn, 0);
    k_adj_update<<<(m.nc + 255) / 256, 256, 0, st>>>(m, W, F, pf, Wn);
}

void launch_adj_reverse(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W,
                        const double* rho_p, double dt, const double* theta, const AdjO2& o2, const double* lam_next,
                        double* lam, double* wbar, double* thbar, double* th_out, cudaStream_t st) {
    const int g = (m.nf + 127) / 128;
    if (p.order == 2) k_adj_grad<<<grad_grid(m), 128, 0, st>>>(m, p, ap, W, rho_p, theta, o2.phi, 0, o2.gW, o2.gH);
    if (p.order == 2)
        k_adj_face<true><<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, o2.gW, o2.gH, lam_next, wbar, o2.gbar, thbar);
    else
        k_adj_face<false><<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, o2.gW, o2.gH, lam_next, wbar, o2.gbar, thbar);
    if (p.order == 2) k_adj_gg<<<(m.nc + 255) / 256, 256, 0, st>>>(m, o2.phi, o2.gbar, o2.gg);
    k_adj_cell<<<(m.nc + 255) / 256, 256, 0, st>>>(m, p, ap, W, theta, lam_next, wbar, o2.gg, lam, o2.thc);
    k_adj_sum<<<1, 256, 0, st>>>(thbar, m.nf, 3, th_out, 0);
    if (p.order == 2) k_adj_sum<<<1, 256, 0, st>>>(o2.thc, m.nc, 3, th_out, 1);
}

}  // namespace ugkwp
