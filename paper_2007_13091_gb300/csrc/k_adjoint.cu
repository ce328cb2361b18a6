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

__device__ __forceinline__ bool listed_face(const DevMesh& m, const AdjParams& ap, int f) {
    const int nb = m.f_nbr[f];
    return nb < 0 && ap.b[m.bf_tag[-1 - nb]].listed;
}

// ---- forward: fluxes and the functional's face terms at theta
__global__ void __launch_bounds__(128) k_adj_fwd_flux(DevMesh m, DevParams P, AdjParams ap, const double* W,
                                                      const double* rho_p, double dt, const double* theta, double* F,
                                                      double* jf) {
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
        face_flux<double>(m, P, ap, f, WL, rho_p[o], WR, nb >= 0 ? rho_p[nb] : 0.0, th, dt, Fv);
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

// out[c] = sum_j x[c n + j] for c < ncomp (one block, fixed order per thread)
__global__ void k_adj_sum(const double* x, int n, int ncomp, double* out) {
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
        if (threadIdx.x == 0) out[c] = sh[0];
        __syncthreads();
    }
}

// ---- reverse: per face, g_f and its products with the local Jacobians
__global__ void __launch_bounds__(128) k_adj_face(DevMesh m, DevParams P, AdjParams ap, const double* W,
                                                  const double* rho_p, double dt, const double* theta,
                                                  const double* lam_next, double* wbar, double* thbar) {
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

__global__ void k_adj_cell(DevMesh m, const double* lam_next, const double* wbar, double* lam) {
    const int nc = m.nc, nf = m.nf;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const int own = m.cfs[i];
    for (int q = 0; q < 5; ++q) {
        double a = lam_next[(size_t)q * nc + i];
        for (int k = 0; k < 4; ++k) {
            const int f = m.cf[k * nc + i];
            a += wbar[(size_t)(((own >> k) & 1) ? q : 5 + q) * nf + f];
        }
        lam[(size_t)q * nc + i] = a;
    }
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

void launch_adj_forward(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W, const double* rho_p,
                        const double* pf, double dt, const double* theta, double* F, double* jf, double* Jn,
                        double* Wn, cudaStream_t st) {
    const int g = (m.nf + 127) / 128;
    k_adj_fwd_flux<<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, F, jf);
    k_adj_sum<<<1, 256, 0, st>>>(jf, m.nf, 1, Jn);
    k_adj_update<<<(m.nc + 255) / 256, 256, 0, st>>>(m, W, F, pf, Wn);
}

void launch_adj_reverse(const DevMesh& m, const DevParams& p, const AdjParams& ap, const double* W,
                        const double* rho_p, double dt, const double* theta, const double* lam_next, double* lam,
                        double* wbar, double* thbar, double* th_out, cudaStream_t st) {
    const int g = (m.nf + 127) / 128;
    k_adj_face<<<g, 128, 0, st>>>(m, p, ap, W, rho_p, dt, theta, lam_next, wbar, thbar);
    k_adj_cell<<<(m.nc + 255) / 256, 256, 0, st>>>(m, lam_next, wbar, lam);
    k_adj_sum<<<1, 256, 0, st>>>(thbar, m.nf, 3, th_out);
}

}  // namespace ugkwp
