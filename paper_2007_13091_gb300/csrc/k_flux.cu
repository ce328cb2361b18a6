// a4: time-integrated wave flux per face, F = F^eq + F^{fr,wave} (per unit
// area, normal from owner to neighbour), first-order reconstruction.
//
//  * W0 from the compatibility condition with the upwind initial state
//    (Sec. 2.1): W0 = rho_L <psi>_{u.n>0, L} + rho_R <psi>_{u.n<0, R};
//  * F^eq = q1 int u.n g0 psi (g_x = g_t = 0 at first order);
//  * F^{fr,wave} = (q4 - dt e^{-dt/tau}) int u.n g0^h psi (Sec. 2.3) with the
//    upwind hydrodynamic Maxwellian g0^h = (rho^h/rho) g of each side;
//  * tau at the face = mu(T0)/p0 + C2 |pL - pR|/|pL + pR| dt (Sec. 2.4 (d));
//  * q1..q5 are the time integrals of c1..c5 (Sec. 2.1), evaluated by their
//    power series in dt/tau below 1 and in closed form above;
//  * boundaries: diffuse wall (Sec. 2.4 (e), zero net wave mass flux), mirror
//    ghost for specular planes, all-hydrodynamic ghosts for far field and
//    zero-gradient outflow (their incoming half carries q4: no particles are
//    emitted from a ghost).
// Maxwellian moments use the recurrence <u^{k+2}> = U <u^{k+1}> + (k+1)/(2 lambda) <u^k>.
#include "ugkwp_internal.hpp"

namespace ugkwp {

namespace {

constexpr double PI = 3.14159265358979323846;

struct Side {
    double rho, rhoh, Un, Ut[3], lam, p, rl;  // rl = 1/sqrt(lambda)
};

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Primitive state in the face frame; two divisions (1/rho, rho/p).
__device__ __forceinline__ Side make_side(const double* W, double rhoh, const double* n) {
    Side s;
    s.rho = W[0];
    const double ir = 1.0 / s.rho;
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    s.p = (W[4] - 0.5 * s.rho * dot3(U, U)) * (2.0 / 3.0);
    s.lam = 0.5 * s.rho / s.p;
    s.rl = rsqrt(s.lam);
    s.rhoh = rhoh;
    s.Un = dot3(U, n);
    for (int c = 0; c < 3; ++c) s.Ut[c] = U[c] - s.Un * n[c];
    return s;
}

// <u_n^k>, k = 0..3, of the normalised Maxwellian over the half space `half`
// (rl = 1/sqrt(lambda)).
__device__ __forceinline__ void moments(double Un, double lam, double rl, int half, double M[4]) {
    const double h = 0.5 * rl * rl;  // 1/(2 lambda)
    if (half == 0) {
        M[0] = 1.0;
        M[1] = Un;
    } else {
        const double a = lam * rl * Un;  // sqrt(lambda) Un
        const double edge = 0.5 * exp(-a * a) * rl * 0.56418958354775628695;  // 1/sqrt(pi)
        if (half > 0) { M[0] = 0.5 * erfc(-a); M[1] = Un * M[0] + edge; }
        else          { M[0] = 0.5 * erfc(a);  M[1] = Un * M[0] - edge; }
    }
    M[2] = Un * M[1] + h * M[0];
    M[3] = Un * M[2] + 2.0 * h * M[1];
}

// G = int_{half} u.n g psi du and H = int_{half} g psi du for a unit-density
// Maxwellian (Un n + Ut, lambda).
__device__ __forceinline__ void flux_moments(double Un, const double* Ut, const double* n, double lam, double rl,
                                             int half, double G[5], double H[5]) {
    double M[4];
    moments(Un, lam, rl, half, M);
    const double tv = dot3(Ut, Ut) + rl * rl;  // |Ut|^2 + 1/lambda
    G[0] = M[1];
    H[0] = M[0];
    for (int c = 0; c < 3; ++c) {
        G[1 + c] = M[2] * n[c] + M[1] * Ut[c];
        H[1 + c] = M[1] * n[c] + M[0] * Ut[c];
    }
    G[4] = 0.5 * (M[3] + M[1] * tv);
    H[4] = 0.5 * (M[2] + M[0] * tv);
}

__constant__ double c_inv_k[31] = {
    0.0, 1.0, 1.0 / 2, 1.0 / 3, 1.0 / 4, 1.0 / 5, 1.0 / 6, 1.0 / 7, 1.0 / 8, 1.0 / 9, 1.0 / 10,
    1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19, 1.0 / 20,
    1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29, 1.0 / 30};

// q1, q4 and a4 = q4 - dt e^{-dt/tau} (the coefficients of the first-order flux).
__device__ __forceinline__ void time_coeffs(double dt, double tau, double& q1, double& q4, double& a4) {
    const double x = dt / tau;
    if (x < 1.0) {
        // power series in x; stop once k x^k/k! falls below 2^-60 x^2 (the
        // smallest leading term, of q1 and a4)
        const double stop = x * x * 0x1p-60;
        double term = 1.0, s1 = 0.0, s4 = 0.0, sa = 0.0;
#pragma unroll 1
        for (int k = 1; k <= 30; ++k) {
            term = term * x * c_inv_k[k];
            const double sg = (k & 1) ? -1.0 : 1.0;  // (-1)^k
            if (k >= 2) s1 += sg * term;
            s4 -= sg * term;
            if (k >= 2) sa += sg * (double)(k - 1) * term;
            if (k >= 3 && term * (double)k < stop) break;
        }
        q1 = tau * s1;
        q4 = tau * s4;
        a4 = tau * sa;
    } else {
        const double e = exp(-x);
        const double ph = -expm1(-x);
        q1 = dt - tau * ph;
        q4 = tau * ph;
        a4 = q4 - dt * e;
    }
}

__device__ void interior_flux(const Side& L, const Side& R, bool ghost_hydro, const double* n, double dt,
                              const DevParams& p, double inv_Tref, double F[5]) {
    double GL[5], HL[5], GR[5], HR[5];
    flux_moments(L.Un, L.Ut, n, L.lam, L.rl, +1, GL, HL);
    flux_moments(R.Un, R.Ut, n, R.lam, R.rl, -1, GR, HR);
    double W0[5];
    for (int q = 0; q < 5; ++q) W0[q] = L.rho * HL[q] + R.rho * HR[q];
    const double rho0 = W0[0];
    const double ir0 = 1.0 / rho0;
    const double U0[3] = {W0[1] * ir0, W0[2] * ir0, W0[3] * ir0};
    const double p0 = (W0[4] - 0.5 * rho0 * dot3(U0, U0)) * (2.0 / 3.0);
    const double ip0 = 1.0 / p0;
    const double lam0 = 0.5 * rho0 * ip0;
    const double T0 = p0 * ir0 / p.R;
    double tau = p.mu_ref * exp(p.omega * log(T0 * inv_Tref)) * ip0;
    if (p.C2 > 0.0) tau += p.C2 * fabs(L.p - R.p) / fabs(L.p + R.p) * dt;
    double q1, q4, a4;
    time_coeffs(dt, tau, q1, q4, a4);
    // full-range moments of g0: the Euler flux of W0
    const double Un0 = dot3(U0, n);
    const double E0 = W0[4];
    double Feq[5];
    Feq[0] = rho0 * Un0;
    for (int c = 0; c < 3; ++c) Feq[1 + c] = rho0 * Un0 * U0[c] + p0 * n[c];
    Feq[4] = Un0 * (E0 + p0);
    (void)lam0;
    const double cR = ghost_hydro ? q4 : a4;
    for (int k = 0; k < 5; ++k) F[k] = q1 * Feq[k] + a4 * (L.rhoh * GL[k]) + cR * (R.rhoh * GR[k]);
}

__global__ void __launch_bounds__(256) k_face_flux(DevMesh m, DevState s, DevParams p) {
    const int nc = m.nc, nf = m.nf;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf) return;
    const int f = m.face_order[t];  // interior faces first, then boundary faces by type
    const double dt = s.dt[0];
    const double inv_Tref = 1.0 / p.T_ref;
    const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
    const int o = m.f_own[f], nb = m.f_nbr[f];
    double WL[5];
    for (int q = 0; q < 5; ++q) WL[q] = s.W[(size_t)q * nc + o];
    const Side L = make_side(WL, s.rhoh[o], n);
    double F[5];
    if (nb >= 0) {
        double WR[5];
        for (int q = 0; q < 5; ++q) WR[q] = s.W[(size_t)q * nc + nb];
        const Side R = make_side(WR, s.rhoh[nb], n);
        interior_flux(L, R, false, n, dt, p, inv_Tref, F);
    } else {
        const DevBc& bc = p.bc[m.bf_tag[-1 - nb]];
        if (bc.type == UGKWP_BC_DIFFUSE_WALL) {
            double q1, q4, a4;
            time_coeffs(dt, s.tau[o], q1, q4, a4);
            double GL[5], HL[5], Gin[5];
            flux_moments(L.Un, L.Ut, n, L.lam, L.rl, +1, GL, HL);
            for (int k = 0; k < 5; ++k) Gin[k] = q1 * (L.rho * GL[k]) + a4 * (L.rhoh * GL[k]);
            const double lamw = 1.0 / (2.0 * p.R * bc.T_w);
            const double Uwn = dot3(bc.U_w, n);
            double Uwt[3];
            for (int c = 0; c < 3; ++c) Uwt[c] = bc.U_w[c] - Uwn * n[c];
            double Gw[5], Hw[5];
            flux_moments(Uwn, Uwt, n, lamw, rsqrt(lamw), -1, Gw, Hw);
            const double rhow = -Gin[0] / (dt * Gw[0]);
            for (int k = 0; k < 5; ++k) F[k] = Gin[k] + dt * rhow * Gw[k];
        } else if (bc.type == UGKWP_BC_SPECULAR) {
            Side R = L;
            R.Un = -L.Un;
            double Ff[5];
            interior_flux(L, R, false, n, dt, p, inv_Tref, Ff);
            const double fn = Ff[1] * n[0] + Ff[2] * n[1] + Ff[3] * n[2];
            F[0] = 0.0;
            F[4] = 0.0;
            for (int c = 0; c < 3; ++c) F[1 + c] = fn * n[c];
        } else {
            Side R = (bc.type == UGKWP_BC_FARFIELD) ? make_side(bc.W_in, bc.W_in[0], n) : L;
            R.rhoh = R.rho;
            interior_flux(L, R, true, n, dt, p, inv_Tref, F);
        }
    }
    for (int q = 0; q < 5; ++q) s.F[(size_t)q * nf + f] = F[q];
}

}  // namespace

void launch_face_flux(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    k_face_flux<<<(m.nf + 255) / 256, 256, 0, st>>>(m, s, p);
}

}  // namespace ugkwp
