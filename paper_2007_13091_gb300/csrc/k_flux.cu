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

// The second-order wave kernels are bound by the FP64 pipe, which a few warps
// per SM saturate; they run as persistent grids (by default one block per SM,
// see LaunchCfg) so that the particle kernels running beside them keep most of
// each SM's registers and warp slots.
#ifndef UGKWP_WAVE_THREADS
#define UGKWP_WAVE_THREADS 128
#endif
#ifndef UGKWP_WAVE_MIN_BLOCKS
#define UGKWP_WAVE_MIN_BLOCKS 1
#endif

namespace ugkwp {

namespace {

struct Side {
    double rho, rhoh, Un, Ut[3], lam, p, rl;  // rl = 1/sqrt(lambda)
};

// Constants of K internal degrees of freedom (rho E = rho |U|^2/2 + (3+K)/2 p,
// <|xi|^2> = K theta, <|xi|^4> = K (K+2) theta^2, theta = 1/(2 lambda)); for
// K = 0 each is the monatomic literal (2/3, 4/3, 1/3, 3, 5/2, 5, 7) exactly.
struct KC {
    double K, c23, c43, c13, e3, e5h, e5, e7;
};
__device__ __forceinline__ KC kconst(int K) {
    KC k;
    k.K = (double)K;
    k.c23 = 2.0 / (3.0 + k.K);
    k.c43 = 4.0 / (3.0 + k.K);
    k.c13 = 1.0 / (3.0 + k.K);
    k.e3 = 3.0 + k.K;
    k.e5h = 0.5 * (5.0 + k.K);
    k.e5 = 5.0 + k.K;
    k.e7 = 7.0 + k.K;
    return k;
}

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Primitive state in the face frame; two divisions (1/rho, rho/p).
__device__ __forceinline__ Side make_side(const double* W, double rhoh, const double* n, const KC& kc) {
    Side s;
    s.rho = W[0];
    const double ir = 1.0 / s.rho;
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    s.p = (W[4] - 0.5 * s.rho * dot3(U, U)) * kc.c23;
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
                                             int half, const KC& kc, double G[5], double H[5]) {
    double M[4];
    moments(Un, lam, rl, half, M);
    const double tv = (dot3(Ut, Ut) + rl * rl) + kc.K * (0.5 * rl * rl);  // |Ut|^2 + 1/lambda + <|xi|^2>
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
    // ghost_hydro: R is a far-field ghost emitting no particles; p.gks: no
    // particles at all (both halves of the free transport carry q4)
    double GL[5], HL[5], GR[5], HR[5];
    const KC kc = kconst(p.K);
    flux_moments(L.Un, L.Ut, n, L.lam, L.rl, +1, kc, GL, HL);
    flux_moments(R.Un, R.Ut, n, R.lam, R.rl, -1, kc, GR, HR);
    double W0[5];
    for (int q = 0; q < 5; ++q) W0[q] = L.rho * HL[q] + R.rho * HR[q];
    const double rho0 = W0[0];
    const double ir0 = 1.0 / rho0;
    const double U0[3] = {W0[1] * ir0, W0[2] * ir0, W0[3] * ir0};
    const double p0 = (W0[4] - 0.5 * rho0 * dot3(U0, U0)) * kc.c23;
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
    const double cL = p.gks ? q4 : a4;
    const double cR = (ghost_hydro || p.gks) ? q4 : a4;
    for (int k = 0; k < 5; ++k) F[k] = q1 * Feq[k] + cL * (L.rhoh * GL[k]) + cR * (R.rhoh * GR[k]);
}

// ------------------------------------------------------------- order 2
// a3: least-squares gradients over the 4 face neighbours (host-precomputed
// coefficients c_k, ghosts mirrored across boundary faces) limited with
// Venkatakrishnan's function, per conservative component and for rho^h.

// Venkatakrishnan's function of the allowed difference d1 and the extrapolated
// difference d2 (same sign, d2 != 0) as the ratio num/den with den > 0:
// num/den = ((d1^2 + eps^2) d2 + 2 d2^2 d1) / (d2 (d1^2 + 2 d2^2 + d1 d2 + eps^2)).
// d1^2 + d1 d2 + 2 d2^2 > 0 for d2 != 0, so den has the sign of d2.
__device__ __forceinline__ void venkat_ratio(double d1, double d2, double eps2, double& num, double& den) {
    num = (d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1;
    den = d2 * (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
    if (den < 0.0) { num = -num; den = -den; }
}

// Limited gradient of quantity q (0..4: W, 5: rho^h) of cell i.
__device__ __forceinline__ void gradient_of(const DevMesh& m, const DevState& s, const DevParams& p, int i, int q) {
    const int nc = m.nc;
    const double self = q < 5 ? s.W[(size_t)q * nc + i] : s.rhoh[i];
    // the neighbour across each local face, from the tet's tracking record
    // (neighbour << 2 | its local face, or -1 - boundary face): one load
    // instead of a face index and then its cells
    const int4 nbv = m.trk_f ? m.trk_f[i].nb : m.trk_d[i].nb;
    double val[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ck = k == 0 ? nbv.x : k == 1 ? nbv.y : k == 2 ? nbv.z : nbv.w;
        const int other = ck >= 0 ? ck >> 2 : ck;
        if (other >= 0) {
            val[k] = q < 5 ? s.W[(size_t)q * nc + other] : s.rhoh[other];
        } else {
            const int b = -1 - other;
            const DevBc& bc = p.bc[m.bf_tag[b]];
            val[k] = self;
            if (bc.type == UGKWP_BC_SPECULAR && q >= 1 && q <= 3) {
                const int nbf = m.nbf;
                double n[3];
                for (int d = 0; d < 3; ++d) n[d] = m.bf_n[(size_t)d * nbf + b];
                const double mn = s.W[(size_t)nc + i] * n[0] + s.W[(size_t)2 * nc + i] * n[1] + s.W[(size_t)3 * nc + i] * n[2];
                val[k] = self - 2.0 * mn * n[q - 1];
            } else if (bc.type == UGKWP_BC_FARFIELD) {
                val[k] = q < 5 ? bc.W_in[q] : bc.W_in[0];
            }
        }
    }
    const double eps2 = m.eps2[i];
    double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int d = 0; d < 3; ++d) g[d] += m.lsq_c[(size_t)(3 * k + d) * nc + i] * (val[k] - self);
    double vmax = self, vmin = self;
#pragma unroll
    for (int k = 0; k < 4; ++k) { vmax = fmax(vmax, val[k]); vmin = fmin(vmin, val[k]); }
    // phi = min(1, min_k num_k/den_k), compared by cross products (den > 0)
    // so that only the chosen ratio is divided
    double bn = 1.0, bd = 1.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double d2 = g[0] * m.lsq_dxf[(size_t)(3 * k) * nc + i] + g[1] * m.lsq_dxf[(size_t)(3 * k + 1) * nc + i] +
                          g[2] * m.lsq_dxf[(size_t)(3 * k + 2) * nc + i];
        if (d2 == 0.0) continue;
        double num, den;
        venkat_ratio(d2 > 0.0 ? vmax - self : vmin - self, d2, eps2, num, den);
        if (num * bd < bn * den) { bn = num; bd = den; }
    }
    const double phi = bn / bd;
    for (int d = 0; d < 3; ++d) {
        if (q < 5) s.gradW[(size_t)(3 * q + d) * nc + i] = phi * g[d];
        else s.gradH[(size_t)d * nc + i] = phi * g[d];
    }
}

// One thread per (quantity, cell), quantity-major so that neighbouring threads
// read neighbouring cells of one array.
__device__ __forceinline__ void gradients_body(const DevMesh& m, const DevState& s, const DevParams& p, Blk bk) {
    const int nc = m.nc;
    const long long n = 6LL * nc;
    for (long long t = (long long)bk.id * blockDim.x + threadIdx.x; t < n; t += (long long)bk.n * blockDim.x) {
        const int q = (int)(t / nc);
        gradient_of(m, s, p, (int)(t - (long long)q * nc), q);
    }
}
__global__ void __launch_bounds__(128) k_gradients(DevMesh m, DevState s, DevParams p) {
    gradients_body(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// Moment tables of a unit Maxwellian in a face frame: <u^k> (normal, over the
// half space `half` or all u) and <v^k>, <w^k> (tangential, full), k = 0..6.
// x1 = <|xi|^2>, x2 = <|xi|^4> - <|xi|^2>^2 = 2 K theta^2 (internal degrees of freedom)
struct Tab { double n[7], v[7], w[7], x1, x2; };

__device__ __forceinline__ void gauss_mom(double mean, double h, double* M) {  // h = 1/(2 lambda)
    M[0] = 1.0;
    M[1] = mean;
#pragma unroll
    for (int k = 0; k < 5; ++k) M[k + 2] = mean * M[k + 1] + (double)(k + 1) * h * M[k];
}

__device__ __forceinline__ void make_tab(const double* U, double lam, double rl, int half, const KC& kc, Tab& T) {
    const double h = 0.5 * rl * rl;
    T.x1 = kc.K * h;
    T.x2 = 2.0 * kc.K * h * h;
    if (half == 0) {
        gauss_mom(U[0], h, T.n);
    } else {
        const double a = lam * rl * U[0];
        const double edge = 0.5 * exp(-a * a) * rl * 0.56418958354775628695;
        T.n[0] = half > 0 ? 0.5 * erfc(-a) : 0.5 * erfc(a);
        T.n[1] = U[0] * T.n[0] + (half > 0 ? edge : -edge);
#pragma unroll
        for (int k = 0; k < 5; ++k) T.n[k + 2] = U[0] * T.n[k + 1] + (double)(k + 1) * h * T.n[k];
    }
    gauss_mom(U[1], h, T.v);
    gauss_mom(U[2], h, T.w);
}

// out_k = < u^AL v^BE w^GA (a.psi) psi_k >, psi = (1, u, v, w, (|u|^2 + |xi|^2)/2).
// With a.psi = A_u(u) + A_v(v) + A_w(w) + a4 |xi|^2/2, A_u = a0 + a1 u + a4 u^2/2,
// A_v = a2 v + a4 v^2/2, A_w = a3 w + a4 w^2/2, every moment factorises into
// 1D tables: <u^x v^y w^z a.psi> = NA_x v_y w_z + n_x (VA_y w_z + v_y WA_z),
// the xi part averaged into a0 (a0 + a4 <|xi|^2>/2) and, for psi_4, the
// moment <|xi|^2 a.psi>/2 = (x1 SS_000 + a4/2 x2 n v w)/2.
template <int AL, int BE, int GA>
__device__ __forceinline__ void apsi(const Tab& T, const double* a, double out[5]) {
    const double h4 = 0.5 * a[4];
    const double a0 = a[0] + h4 * T.x1;
    double NA[3], VA[3], WA[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        NA[i] = a0 * T.n[AL + i] + a[1] * T.n[AL + i + 1] + h4 * T.n[AL + i + 2];
        VA[i] = a[2] * T.v[BE + i + 1] + h4 * T.v[BE + i + 2];
        WA[i] = a[3] * T.w[GA + i + 1] + h4 * T.w[GA + i + 2];
    }
#define SS(x, y, z) (NA[x] * T.v[BE + (y)] * T.w[GA + (z)] + \
                     T.n[AL + (x)] * (VA[y] * T.w[GA + (z)] + T.v[BE + (y)] * WA[z]))
    out[0] = SS(0, 0, 0);
    out[1] = SS(1, 0, 0);
    out[2] = SS(0, 1, 0);
    out[3] = SS(0, 0, 1);
    out[4] = 0.5 * ((SS(2, 0, 0) + SS(0, 2, 0) + SS(0, 0, 2)) +
                    (T.x1 * out[0] + h4 * T.x2 * (T.n[AL] * T.v[BE] * T.w[GA])));
#undef SS
}

// out_k = < u^AL psi_k > (a = e_0).
template <int AL>
__device__ __forceinline__ void psi_mom(const Tab& T, double out[5]) {
    out[0] = T.n[AL];
    out[1] = T.n[AL + 1];
    out[2] = T.n[AL] * T.v[1];
    out[3] = T.n[AL] * T.w[1];
    out[4] = 0.5 * (T.n[AL + 2] + T.n[AL] * ((T.v[2] + T.w[2]) + T.x1));
}

// <u_n u_d (a.psi) psi> for frame direction d (0 normal, 1 t1, 2 t2)
__device__ __forceinline__ void slope_mom(const Tab& T, int d, const double* a, double out[5]) {
    if (d == 0) apsi<2, 0, 0>(T, a, out);
    else if (d == 1) apsi<1, 1, 0>(T, a, out);
    else apsi<1, 0, 1>(T, a, out);
}

// Micro slope a with <psi psi^T> a = b for the unit Maxwellian (U, lambda),
// in closed form: with theta = 1/(2 lambda), R_i = b_i - U_i b_0,
// R_4 = 2 b_4 - (|U|^2 + 3 theta) b_0:  a_4 = 4 lambda^2/3 (R_4 - 2 U.R),
// a_i = 2 lambda R_i - U_i a_4,  a_0 = b_0 - U.a - a_4 (|U|^2 + 3 theta)/2.
__device__ __forceinline__ void micro(const double* U, double lam, double th, const double* b, double* a,
                                      const KC& kc) {
    const double R1 = b[1] - U[0] * b[0], R2 = b[2] - U[1] * b[0], R3 = b[3] - U[2] * b[0];
    const double U2 = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
    const double R4 = 2.0 * b[4] - (U2 + kc.e3 * th) * b[0];
    a[4] = kc.c43 * lam * lam * (R4 - 2.0 * (U[0] * R1 + U[1] * R2 + U[2] * R3));
    a[1] = 2.0 * lam * R1 - U[0] * a[4];
    a[2] = 2.0 * lam * R2 - U[1] * a[4];
    a[3] = 2.0 * lam * R3 - U[2] * a[4];
    a[0] = b[0] - (U[0] * a[1] + U[1] * a[2] + U[2] * a[3]) - 0.5 * a[4] * (U2 + kc.e3 * th);
}

// All time coefficients: q1, q2, q3, q4, a4, a5 in closed form from one
// expm1.  Where x = dt/tau is small the differences cancel, but their absolute
// errors stay at rounding level of dt (q1, q4, a4) and dt^2 (q2, q3, a5), the
// scales at which they enter the flux.
struct QC { double q1, q2, q3, q4, q5, a4, a5; };
__device__ __forceinline__ QC time_coeffs_all(double dt, double tau) {
    QC c;
    const double em1 = expm1(-dt / tau);  // e^{-dt/tau} - 1
    const double e = 1.0 + em1;
    const double tdt = tau * dt;
    c.q4 = -tau * em1;
    c.q1 = dt - c.q4;
    c.a4 = c.q4 - dt * e;
    c.q2 = 2.0 * tau * c.q4 - tdt - tdt * e;
    c.q3 = 0.5 * dt * dt - tdt + tau * c.q4;
    c.q5 = tdt * e - tau * c.q4;
    c.a5 = c.q5 + 0.5 * dt * dt * e;
    return c;
}

// Face frame rows n, t1, t2 (t1 = e_a x n / |.| for the axis of smallest |n_a|).
__device__ __forceinline__ void face_frame(const double* n, double R[3][3]) {
    int ax = 0;
    if (fabs(n[1]) < fabs(n[ax])) ax = 1;
    if (fabs(n[2]) < fabs(n[ax])) ax = 2;
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

// Slopes along frame direction dd of the frame-rotated W, from a cell gradient.
__device__ __forceinline__ void frame_slope(const double* gW, int nc, int c, const double R[3][3], int dd, double out[5]) {
    double g[5];
#pragma unroll
    for (int q = 0; q < 5; ++q)
        g[q] = gW[(size_t)(3 * q) * nc + c] * R[dd][0] + gW[(size_t)(3 * q + 1) * nc + c] * R[dd][1] +
               gW[(size_t)(3 * q + 2) * nc + c] * R[dd][2];
    out[0] = g[0];
    for (int j = 0; j < 3; ++j) out[1 + j] = R[j][0] * g[1] + R[j][1] * g[2] + R[j][2] * g[3];
    out[4] = g[4];
}

// Equilibrium slope terms in closed form.  For the unit-density Maxwellian
// (U, theta = 1/(2 lambda)) and a micro slope a with <psi psi^T> a = b, the
// product (a.psi) g is the derivative of g(W) along b, so every slope moment is
// the derivative of a Maxwellian moment along b, with
// d rho = b0, dU = b_{1..3} - U b0, d theta = (2 b4 - (|U|^2 + 3 theta) b0 - 2 U.dU)/3:
//   <u_D (a.psi) psi>     = dF_D(b), F_D the Euler flux along D,
//   <u_n u_D (a.psi) psi> = dQ_D(b), Q_D = <u_n u_D psi g> with
//   <u_i u_j> = U_i U_j + theta d_ij,
//   <u_i u_j u_k> = U_i U_j U_k + theta (U_i d_jk + U_j d_ik + U_k d_ij),
//   <u_i u_j |u|^2/2> = (U_i U_j (|U|^2 + 7 theta) + d_ij theta (|U|^2 + 5 theta))/2.
// The face frame has the normal as direction 0.
struct DPrim { double dr, dU[3], dth, UdU; };

__device__ __forceinline__ DPrim dprim(const double* U, double th, double U2, const double* b, const KC& kc) {
    DPrim q;
    q.dr = b[0];
    for (int j = 0; j < 3; ++j) q.dU[j] = b[1 + j] - U[j] * b[0];
    q.UdU = U[0] * q.dU[0] + U[1] * q.dU[1] + U[2] * q.dU[2];
    q.dth = ((2.0 * b[4] - (U2 + kc.e3 * th) * b[0]) - 2.0 * q.UdU) * kc.c13;
    return q;
}

// dF_D(b) (Euler flux Jacobian along frame direction D applied to b)
template <int D>
__device__ __forceinline__ void euler_jac(const double* U, double th, double U2, const double* b, const DPrim& q,
                                          const KC& kc, double out[5]) {
    out[0] = b[1 + D];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        double v = q.dr * (U[D] * U[j]) + q.dU[D] * U[j] + U[D] * q.dU[j];
        if (j == D) v += q.dr * th + q.dth;
        out[1 + j] = v;
    }
    out[4] = b[1 + D] * (0.5 * U2 + kc.e5h * th) + U[D] * (q.UdU + kc.e5h * q.dth);
}

// dQ_D(b) = <u_n u_D (a.psi) psi>
template <int D>
__device__ __forceinline__ void q_jac(const double* U, double th, double U2, const DPrim& q, const KC& kc,
                                      double out[5]) {
    const double un_ud = U[0] * U[D];
    const double d_un_ud = q.dU[0] * U[D] + U[0] * q.dU[D];
    out[0] = q.dr * un_ud + d_un_ud;
    if (D == 0) out[0] += q.dr * th + q.dth;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // Q = U_n U_D U_j + theta (U_n d_Dj + U_D d_nj + U_j d_nD)
        double s = 0.0, ds = 0.0;  // sum of the delta-selected velocities and its derivative
        if (D == j) { s += U[0]; ds += q.dU[0]; }
        if (j == 0) { s += U[D]; ds += q.dU[D]; }
        if (D == 0) { s += U[j]; ds += q.dU[j]; }
        out[1 + j] = q.dr * (un_ud * U[j] + th * s) + d_un_ud * U[j] + un_ud * q.dU[j] + q.dth * s + th * ds;
    }
    // <u_i u_j (|u|^2 + |xi|^2)> = U_i U_j (|U|^2 + (7+K) theta) + d_ij theta (|U|^2 + (5+K) theta)
    const double A = U2 + kc.e7 * th;
    double v = q.dr * (0.5 * un_ud * A) + 0.5 * (d_un_ud * A + un_ud * (2.0 * q.UdU + kc.e7 * q.dth));
    if (D == 0) {
        const double Bq = U2 + kc.e5 * th;
        v += q.dr * (0.5 * th * Bq) + 0.5 * (q.dth * Bq + th * (2.0 * q.UdU + kc.e5 * q.dth));
    }
    out[4] = v;
}

// One side of an interior face at second order, in the face frame: the
// reconstructed state (first order if not positive), its half-space moments
// H = <psi>, G = <u_n psi>, the slope part S = sum_d <u_n u_d (a^h_d.psi) psi>
// of its hydrodynamic wave (a^h_d solved from grad_d W^h, W^h = (rho^h/rho) W),
// and half of its frame slopes of W (the equilibrium slope averages both sides).
struct SideOut {
    double rho, rhoh, p;
    double H[5], G[5], S[5];
};

__device__ __forceinline__ SideOut side_o2(const DevMesh& m, const DevState& s, int c, const double* dx,
                                           const double R[3][3], int half, double B[3][5], bool first,
                                           const KC& kc) {
    const int nc = m.nc;
    double Wf[5];
    for (int q = 0; q < 5; ++q)
        Wf[q] = s.W[(size_t)q * nc + c] + s.gradW[(size_t)(3 * q) * nc + c] * dx[0] +
                s.gradW[(size_t)(3 * q + 1) * nc + c] * dx[1] + s.gradW[(size_t)(3 * q + 2) * nc + c] * dx[2];
    double rh = s.rhoh[c] + s.gradH[c] * dx[0] + s.gradH[nc + c] * dx[1] + s.gradH[2 * nc + c] * dx[2];
    double pr = (Wf[4] - 0.5 * (Wf[1] * Wf[1] + Wf[2] * Wf[2] + Wf[3] * Wf[3]) / Wf[0]) * kc.c23;
    const bool o2 = Wf[0] > 0.0 && pr > 0.0;
    if (!o2) {
        for (int q = 0; q < 5; ++q) Wf[q] = s.W[(size_t)q * nc + c];
        rh = s.rhoh[c];
        pr = (Wf[4] - 0.5 * (Wf[1] * Wf[1] + Wf[2] * Wf[2] + Wf[3] * Wf[3]) / Wf[0]) * kc.c23;
    }
    SideOut o;
    double W[5];
    W[0] = Wf[0];
    for (int j = 0; j < 3; ++j) W[1 + j] = R[j][0] * Wf[1] + R[j][1] * Wf[2] + R[j][2] * Wf[3];
    W[4] = Wf[4];
    o.rho = W[0];
    o.rhoh = rh;
    o.p = pr;
    const double ir = 1.0 / W[0];
    const double U[3] = {W[1] * ir, W[2] * ir, W[3] * ir};
    const double lam = 0.5 * W[0] / pr;
    const double rl = rsqrt(lam);
    const double th = 0.5 * rl * rl;
    Tab T;
    make_tab(U, lam, rl, half, kc, T);
    psi_mom<0>(T, o.H);
    psi_mom<1>(T, o.G);
    for (int k = 0; k < 5; ++k) o.S[k] = 0.0;
    if (!o2) {
        if (first) for (int dd = 0; dd < 3; ++dd) for (int q = 0; q < 5; ++q) B[dd][q] = 0.0;
        return o;
    }
    const double ratio = rh * ir;
    for (int dd = 0; dd < 3; ++dd) {
        double dW[5], b[5], a[5], sm[5];
        frame_slope(s.gradW, nc, c, R, dd, dW);
        for (int q = 0; q < 5; ++q) B[dd][q] = first ? 0.5 * dW[q] : B[dd][q] + 0.5 * dW[q];
        const double gh = s.gradH[c] * R[dd][0] + s.gradH[nc + c] * R[dd][1] + s.gradH[2 * nc + c] * R[dd][2];
        const double gr = (gh - ratio * dW[0]) * ir;
        for (int q = 0; q < 5; ++q) b[q] = ratio * dW[q] + W[q] * gr;
        micro(U, lam, th, b, a, kc);
        slope_mom(T, dd, a, sm);
        for (int k = 0; k < 5; ++k) o.S[k] += sm[k];
    }
    return o;
}

__device__ void interior_flux_o2(const DevMesh& m, const DevState& s, const DevParams& p, int f, int o, int nb,
                                 const double* n, double dt, double inv_Tref, double F[5]) {
    const int nc = m.nc;
    double R[3][3];
    face_frame(n, R);
    const int lk = m.f_lk[f];
    double dxL[3], dxR[3];
    for (int d = 0; d < 3; ++d) {
        dxL[d] = m.lsq_dxf[(size_t)(3 * (lk & 3) + d) * nc + o];
        dxR[d] = m.lsq_dxf[(size_t)(3 * ((lk >> 2) & 3) + d) * nc + nb];
    }
    double B[3][5];
    const KC kc = kconst(p.K);
    const SideOut L = side_o2(m, s, o, dxL, R, +1, B, true, kc);
    const SideOut Rs = side_o2(m, s, nb, dxR, R, -1, B, false, kc);
    double W0[5];
    for (int k = 0; k < 5; ++k) W0[k] = L.rho * L.H[k] + Rs.rho * Rs.H[k];
    const double rho0 = W0[0], ir0 = 1.0 / rho0;
    const double U0[3] = {W0[1] * ir0, W0[2] * ir0, W0[3] * ir0};
    const double p0 = (W0[4] - 0.5 * rho0 * dot3(U0, U0)) * kc.c23;
    const double T0 = p0 * ir0 / p.R;
    double tau = p.mu_ref * exp(p.omega * log(T0 * inv_Tref)) / p0;
    if (p.C2 > 0.0) tau += p.C2 * fabs(L.p - Rs.p) / fabs(L.p + Rs.p) * dt;
    const QC qc = time_coeffs_all(dt, tau);
    // free transport of the hydrodynamic wave, upwind, with slopes; without
    // particles (GKS step) the whole free transport, q4 and q5, is the wave's
    const double c4 = p.gks ? qc.q4 : qc.a4, c5 = p.gks ? qc.q5 : qc.a5;
    for (int k = 0; k < 5; ++k)
        F[k] = c4 * (L.rhoh * L.G[k] + Rs.rhoh * Rs.G[k]) + c5 * (L.S[k] + Rs.S[k]);
    // equilibrium part Fe: q1 g0 + q2 u.g_x + q3 g_t, in closed form
    const double th0 = p0 * ir0;
    const double U20 = dot3(U0, U0);
    double Fe[5];
    Fe[0] = qc.q1 * W0[1];
    for (int j = 0; j < 3; ++j) Fe[1 + j] = qc.q1 * (W0[1] * U0[j] + (j == 0 ? p0 : 0.0));
    Fe[4] = qc.q1 * U0[0] * (W0[4] + p0);
    double Wt[5], t5[5];
    {
        const DPrim q = dprim(U0, th0, U20, B[0], kc);
        q_jac<0>(U0, th0, U20, q, kc, t5);
        for (int k = 0; k < 5; ++k) Fe[k] += qc.q2 * t5[k];
        euler_jac<0>(U0, th0, U20, B[0], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] = -t5[k];
    }
    {
        const DPrim q = dprim(U0, th0, U20, B[1], kc);
        q_jac<1>(U0, th0, U20, q, kc, t5);
        for (int k = 0; k < 5; ++k) Fe[k] += qc.q2 * t5[k];
        euler_jac<1>(U0, th0, U20, B[1], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] -= t5[k];
    }
    {
        const DPrim q = dprim(U0, th0, U20, B[2], kc);
        q_jac<2>(U0, th0, U20, q, kc, t5);
        for (int k = 0; k < 5; ++k) Fe[k] += qc.q2 * t5[k];
        euler_jac<2>(U0, th0, U20, B[2], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] -= t5[k];
    }
    {
        const DPrim q = dprim(U0, th0, U20, Wt, kc);
        euler_jac<0>(U0, th0, U20, Wt, q, kc, t5);
        for (int k = 0; k < 5; ++k) Fe[k] += qc.q3 * t5[k];
    }
    if (p.pr_fix != 0.0) {
        // Prandtl-number fix: + (1/Pr - 1) q_n, q_n the heat flux of Fe relative
        // to U0, from its flux moments and its full moments q1 W0 + (q3 - q2) W_t
        // (int psi u.g_x = -W_t, int psi g_t = W_t):
        // q_n = Fe_E - U0.Fe_m + |U0|^2/2 Fe_rho - U0_n (E' - U0.M' + |U0|^2/2 rho')
        double mo[5];
        for (int k = 0; k < 5; ++k) mo[k] = qc.q1 * W0[k] + (qc.q3 - qc.q2) * Wt[k];
        const double qf = (Fe[4] - ((U0[0] * Fe[1] + U0[1] * Fe[2]) + U0[2] * Fe[3])) + 0.5 * U20 * Fe[0];
        const double qm = (mo[4] - ((U0[0] * mo[1] + U0[1] * mo[2]) + U0[2] * mo[3])) + 0.5 * U20 * mo[0];
        Fe[4] += p.pr_fix * (qf - U0[0] * qm);
    }
    for (int k = 0; k < 5; ++k) F[k] += Fe[k];
    // back to the lab frame
    const double Fm[3] = {F[1], F[2], F[3]};
    for (int d = 0; d < 3; ++d) F[1 + d] = Fm[0] * R[0][d] + Fm[1] * R[1][d] + Fm[2] * R[2][d];
}

// First-order g_p sampling (Sec. 2.2), per cell: g_p = g - c (u.grad g + g_t),
// c = tau - dt e^{-dt/tau}/(1 - e^{-dt/tau}), with grad g from the limited
// gradient and g_t from W_t = -sum_d dF_d/dx_d; as a polynomial phi of
// X = (u - U)/sqrt(RT) in g_p = rho N(X)(1 + phi), bounded over |X| <= 5 and
// scaled down where that bound Phi exceeds 1; stores GP_NC values per cell.
__device__ __forceinline__ void gp_coef_body(const DevMesh& m, const DevState& s, const DevParams& p, Blk bk) {
    const int nc = m.nc;
    const int i = bk.id * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double rho = s.prim[i];
    const double U[3] = {s.prim[nc + i], s.prim[2 * nc + i], s.prim[3 * nc + i]};
    const double th = p.R * s.prim[4 * nc + i];
    const double lam = 0.5 / th;
    const double sig = sqrt(th);
    const double U2 = dot3(U, U);
    const double ir = 1.0 / rho;
    const KC kc = kconst(p.K);
    double bd[3][5], a[3][5], Wt[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, t5[5];
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 5; ++q) bd[d][q] = s.gradW[(size_t)(3 * q + d) * nc + i] * ir;
    {
        const DPrim q = dprim(U, th, U2, bd[0], kc);
        euler_jac<0>(U, th, U2, bd[0], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] -= t5[k];
    }
    {
        const DPrim q = dprim(U, th, U2, bd[1], kc);
        euler_jac<1>(U, th, U2, bd[1], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] -= t5[k];
    }
    {
        const DPrim q = dprim(U, th, U2, bd[2], kc);
        euler_jac<2>(U, th, U2, bd[2], q, kc, t5);
        for (int k = 0; k < 5; ++k) Wt[k] -= t5[k];
    }
    double B[5];
    for (int d = 0; d < 3; ++d) micro(U, lam, th, bd[d], a[d], kc);
    micro(U, lam, th, Wt, B, kc);
    // P(u) = B0 + v.u + u^T K u + (h/2)|u|^2 + (|u|^2/2)(beta.u), K[d][j] = a_d,1+j
    double v[3], beta[3];
    const double h = B[4];
    for (int j = 0; j < 3; ++j) {
        v[j] = B[1 + j] + a[j][0];
        beta[j] = a[j][4];
    }
    const double bU = dot3(beta, U);
    double KU[3], UKU = 0.0;
    for (int d = 0; d < 3; ++d) {
        KU[d] = 0.0;
        for (int j = 0; j < 3; ++j) {
            KU[d] += (a[d][1 + j] + a[j][1 + d]) * U[j];
            UKU += U[d] * a[d][1 + j] * U[j];
        }
    }
    double co[13];
    co[0] = B[0] + dot3(v, U) + UKU + 0.5 * h * U2 + 0.5 * U2 * bU;
    for (int d = 0; d < 3; ++d) {
        co[1 + d] = sig * (v[d] + KU[d] + h * U[d] + 0.5 * U2 * beta[d] + bU * U[d]);
        co[10 + d] = 0.5 * sig * sig * sig * beta[d];
    }
    const int qi[6] = {0, 1, 2, 0, 0, 1}, qj[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        const int d = qi[k], j = qj[k];
        co[4 + k] = sig * sig * (0.5 * (a[d][1 + j] + a[j][1 + d]) + 0.5 * (U[d] * beta[j] + U[j] * beta[d]) +
                                 (d == j ? 0.5 * h + 0.5 * bU : 0.0));
    }
    const double dt = s.dt[0];
    const double e = exp(-(dt / s.tau[i]));
    const double c = s.tau[i] - dt * e / (1.0 - e);
    for (int k = 0; k < 13; ++k) co[k] = -c * co[k];
    const double nL = sqrt(co[1] * co[1] + co[2] * co[2] + co[3] * co[3]);
    const double nQ = sqrt(co[4] * co[4] + co[5] * co[5] + co[6] * co[6] + 2.0 * (co[7] * co[7] + co[8] * co[8] + co[9] * co[9]));
    const double nC = sqrt(co[10] * co[10] + co[11] * co[11] + co[12] * co[12]);
    double Phi = fabs(co[0]) + 5.0 * nL + 25.0 * nQ + 125.0 * nC;
    if (Phi > 1.0) {
        for (int k = 0; k < 13; ++k) co[k] = co[k] / Phi;
        Phi = 1.0;
    }
    for (int k = 0; k < 13; ++k) s.gpc[(size_t)k * nc + i] = co[k];
    s.gpc[(size_t)13 * nc + i] = 1.0 + Phi;
}
__global__ void __launch_bounds__(128) k_gp_coef(DevMesh m, DevState s, DevParams p) {
    gp_coef_body(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

__device__ __forceinline__ void face_flux_o1(const DevMesh& m, const DevState& s, const DevParams& p, int t);

// Second-order flux of the interior faces (the first nif entries of face_order),
// then the first-order flux of the boundary faces that follow them.
// With local time steps (GKS step) each face is integrated over the smaller
// step of its cells and stores the mean flux rate F / dt_f.
__device__ __forceinline__ void face_flux_o2_body(const DevMesh& m, const DevState& s, const DevParams& p, Blk bk) {
    const int nf = m.nf;
    const double dt = s.dt[0];
    const double inv_Tref = 1.0 / p.T_ref;
    for (int t = bk.id * blockDim.x + threadIdx.x; t < nf; t += bk.n * blockDim.x) {
        if (t >= m.nif) {  // the boundary faces follow, at first order, in the same grid
            face_flux_o1(m, s, p, t);
            continue;
        }
        const int f = m.face_order[t];
        const int o = m.f_own[f], nb = m.f_nbr[f];
        const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
        const double dtf = p.gks == 2 ? fmin(s.dtc[o], s.dtc[nb]) : dt;
        double F[5];
        interior_flux_o2(m, s, p, f, o, nb, n, dtf, inv_Tref, F);
        if (p.gks == 2)
            for (int q = 0; q < 5; ++q) F[q] = F[q] / dtf;
        for (int q = 0; q < 5; ++q) s.F[(size_t)q * nf + f] = F[q];
    }
}
__global__ void __launch_bounds__(UGKWP_WAVE_THREADS, UGKWP_WAVE_MIN_BLOCKS) k_face_flux_o2(DevMesh m, DevState s, DevParams p) {
    face_flux_o2_body(m, s, p, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// First-order flux of face face_order[t].
__device__ __forceinline__ void face_flux_o1(const DevMesh& m, const DevState& s, const DevParams& p, int t) {
    const int nc = m.nc, nf = m.nf;
    const int f = m.face_order[t];  // interior faces first, then boundary faces by type
    const double inv_Tref = 1.0 / p.T_ref;
    const double n[3] = {m.f_n[f], m.f_n[nf + f], m.f_n[2 * nf + f]};
    const int o = m.f_own[f], nb = m.f_nbr[f];
    // local time steps (GKS step): the smaller step of the face's cells
    const double dt = p.gks == 2 ? (nb >= 0 ? fmin(s.dtc[o], s.dtc[nb]) : s.dtc[o]) : s.dt[0];
    double WL[5];
    for (int q = 0; q < 5; ++q) WL[q] = s.W[(size_t)q * nc + o];
    const KC kc = kconst(p.K);
    const Side L = make_side(WL, s.rhoh[o], n, kc);
    double F[5];
    if (nb >= 0) {
        double WR[5];
        for (int q = 0; q < 5; ++q) WR[q] = s.W[(size_t)q * nc + nb];
        const Side R = make_side(WR, s.rhoh[nb], n, kc);
        interior_flux(L, R, false, n, dt, p, inv_Tref, F);
    } else {
        const DevBc& bc = p.bc[m.bf_tag[-1 - nb]];
        if (bc.type == UGKWP_BC_DIFFUSE_WALL) {
            double q1, q4, a4;
            time_coeffs(dt, s.tau[o], q1, q4, a4);
            double GL[5], HL[5], Gin[5];
            flux_moments(L.Un, L.Ut, n, L.lam, L.rl, +1, kc, GL, HL);
            const double c4 = p.gks ? q4 : a4;
            for (int k = 0; k < 5; ++k) Gin[k] = q1 * (L.rho * GL[k]) + c4 * (L.rhoh * GL[k]);
            const double lamw = 1.0 / (2.0 * p.R * bc.T_w);
            const double Uwn = dot3(bc.U_w, n);
            double Uwt[3];
            for (int c = 0; c < 3; ++c) Uwt[c] = bc.U_w[c] - Uwn * n[c];
            double Gw[5], Hw[5];
            flux_moments(Uwn, Uwt, n, lamw, rsqrt(lamw), -1, kc, Gw, Hw);
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
            Side R = (bc.type == UGKWP_BC_FARFIELD) ? make_side(bc.W_in, bc.W_in[0], n, kc) : L;
            R.rhoh = R.rho;
            interior_flux(L, R, true, n, dt, p, inv_Tref, F);
        }
    }
    if (p.gks == 2)
        for (int q = 0; q < 5; ++q) F[q] = F[q] / dt;
    for (int q = 0; q < 5; ++q) s.F[(size_t)q * nf + f] = F[q];
}

// First-order flux of the faces face_order[first..nf), grid-stride.
__device__ __forceinline__ void face_flux_body(const DevMesh& m, const DevState& s, const DevParams& p, int first, Blk bk) {
    for (int t = first + bk.id * blockDim.x + threadIdx.x; t < m.nf; t += bk.n * blockDim.x)
        face_flux_o1(m, s, p, t);
}
__global__ void __launch_bounds__(256) k_face_flux(DevMesh m, DevState s, DevParams p, int first) {
    face_flux_body(m, s, p, first, Blk{(int)blockIdx.x, (int)gridDim.x});
}

// ---- fused batches: member i of the chunk runs on the blocks
// off[cls][i] .. off[cls][i + 1] - 1.
__device__ __forceinline__ int member_of(const int32_t* off, int n) {
    int lo = 0, hi = n;  // off[lo] <= blockIdx.x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= (int)blockIdx.x) lo = mid;
        else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ Blk member_blk(const int32_t* off, int i) {
    return Blk{(int)blockIdx.x - off[i], off[i + 1] - off[i]};
}
__global__ void __launch_bounds__(128) k_gradients_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_GRAD], c.n);
    gradients_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, member_blk(c.off[BCL_GRAD], i));
}
__global__ void __launch_bounds__(128) k_gp_coef_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_GPC], c.n);
    gp_coef_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, member_blk(c.off[BCL_GPC], i));
}
__global__ void __launch_bounds__(UGKWP_WAVE_THREADS, UGKWP_WAVE_MIN_BLOCKS)
    k_face_flux_o2_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_FLUX_O2], c.n);
    face_flux_o2_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, member_blk(c.off[BCL_FLUX_O2], i));
}
__global__ void __launch_bounds__(256) k_face_flux_b(const __grid_constant__ BatchChunk c) {
    const int i = member_of(c.off[BCL_FLUX], c.n);
    face_flux_body(c.mem[i].m, c.mem[i].s, c.mem[i].p, 0, member_blk(c.off[BCL_FLUX], i));
}

}  // namespace

static int wave_grid(int n, int blocks) {
    const int need = (n + UGKWP_WAVE_THREADS - 1) / UGKWP_WAVE_THREADS;
    return need < blocks ? need : blocks;
}

// A persistent grid of 4 blocks per SM (56 registers at 128 threads): enough
// warps for this latency-bound kernel, and room beside it for the first half
// of the tracking grid.
void launch_gradients(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    const long long need = (6LL * m.nc + 127) / 128;
    const long long cap = 4LL * sm_count();
    k_gradients<<<(int)(need < cap ? need : cap), 128, 0, st>>>(m, s, p);
}

void launch_gp_coef(const DevMesh& m, const DevState& s, const DevParams& p, cudaStream_t st) {
    k_gp_coef<<<blocks_gp_coef(m.nc), 128, 0, st>>>(m, s, p);
}

void launch_face_flux_o2(const DevMesh& m, const DevState& s, const DevParams& p, int blocks, cudaStream_t st) {
    k_face_flux_o2<<<wave_grid(m.nf, blocks), UGKWP_WAVE_THREADS, 0, st>>>(m, s, p);
}

int wave_threads() { return UGKWP_WAVE_THREADS; }

cudaError_t configure_wave_kernels(int carveout) {
    cudaError_t e = cudaSuccess;
    auto set = [&](auto f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    };
    set(k_gradients);
    set(k_gp_coef);
    set(k_face_flux_o2);
    set(k_face_flux);
    set(k_gradients_b);
    set(k_gp_coef_b);
    set(k_face_flux_o2_b);
    set(k_face_flux_b);
    return e;
}

// blocks > 0 bounds the grid (a step of the method: the flux shares the GPU
// with the particle kernels launched beside it); 0: one thread per face.
void launch_face_flux(const DevMesh& m, const DevState& s, const DevParams& p, int first, int blocks,
                      cudaStream_t st) {
    const int need = (m.nf - first + 255) / 256;
    k_face_flux<<<blocks > 0 && blocks < need ? blocks : need, 256, 0, st>>>(m, s, p, first);
}

int blocks_gp_coef(int nc) { return (nc + 127) / 128; }
int gradient_threads() { return 128; }

void launch_gradients_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_gradients_b<<<blocks, 128, 0, st>>>(c);
}
void launch_gp_coef_batch(const BatchChunk& c, int blocks, cudaStream_t st) { k_gp_coef_b<<<blocks, 128, 0, st>>>(c); }
void launch_face_flux_o2_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_face_flux_o2_b<<<blocks, UGKWP_WAVE_THREADS, 0, st>>>(c);
}
void launch_face_flux_batch(const BatchChunk& c, int blocks, cudaStream_t st) {
    k_face_flux_b<<<blocks, 256, 0, st>>>(c);
}

}  // namespace ugkwp
