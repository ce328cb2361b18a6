// Plain CPU oracle of one UGKWP time step on a tetrahedral mesh.
//
// TEST INFRASTRUCTURE ONLY -- see ugkwp_oracle.h.  Written for a reader who
// checks it against the paper (Chen, Zhu, Xu, "A three-dimensional unified
// gas-kinetic wave-particle solver for flow computation in all regimes",
// arXiv 2007.13091): every step cites the section or equation it follows.
// It is single-threaded FP64 (particle state optionally binary32, "mixed"),
// keeps particles in a plain std::vector and runs the steps of the method in
// the order of the particle evolution procedure of Sec. 2.2:
//
//   a1  primitives and relaxation time per cell            (Sec. 2, tau = mu/p)
//   a2  time step                                          (Sec. 2.4 (a))
//   a5  sampling of the collisionless hydrodynamic particles (Sec. 2.4 (b))
//   a6  free-transport time of the remaining particles     (Eq. t_f)
//   a7  ballistic streaming with face-by-face tet tracking (Sec. 2.2)
//   a8  particle flux by counting                          (Eq. F^{fr,p})
//   a9  removal of collisional and exited particles        (Sec. 2.2 step 4)
//   a4  wave flux F^eq + F^{fr,wave} per face              (Sec. 2.1, 2.3, 2.4 (d),(e))
//   a10 conservative update of W                           (Eq. update_macro_variables)
//
// Readings where the paper is silent are listed in the repository design
// notes; each is marked "reading:" below.
//
// Parity unpinned (no pin independent of this code beyond conservation, the
// free-molecular profile and the continuum limit): the upwind reading of the
// wave's free transport in interior_flux, the far-field ghost of
// boundary_flux (all hydrodynamic, emitting no particles), and the
// least-squares weights and limiter constant of limited_gradients (pinned
// only through properties any such choice has: exact gradients of linear
// fields, the limiter's bounds and its relaxation as epsilon grows).
#include "ugkwp_oracle.h"
#include "omath.hpp"
#include "dual.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

namespace orc {

static const double PI = 3.14159265358979323846;

// ------------------------------------------------------------------ ids, tags
// Particle id: (step born : 24 | cell born : 24 | index in cell : 16).
static inline uint64_t make_id(uint64_t step, uint64_t cell, uint64_t k) {
    return (step << 40) | (cell << 16) | k;
}
static inline uint64_t id_step(uint64_t id) { return id >> 40; }
// Random-number purposes (third counter word).
enum { TAG_TF = 1, TAG_SVEL = 2, TAG_SPOS = 3, TAG_WALL = 4, TAG_GP = 5, TAG_SINT = 6, TAG_WINT = 7 };

static inline Ctr4 draw(uint64_t seed, uint64_t a, uint64_t b, uint64_t tag, uint64_t idx) {
    Ctr4 c; c.v[0] = a; c.v[1] = b; c.v[2] = tag; c.v[3] = idx;
    return philox4x64_10(c, seed, 0);
}

// The free-transport-time draw of particle `id` at `step`: Philox4x32-10 with
// counter (id low, id high, step, TAG_TF) and key (seed low, seed high); the
// first two output words form the 64 random bits (word 0 high).
static inline uint64_t draw_tf(uint64_t seed, uint64_t id, uint64_t step) {
    Ctr4x32 c;
    c.v[0] = (uint32_t)id; c.v[1] = (uint32_t)(id >> 32); c.v[2] = (uint32_t)step; c.v[3] = 1u;
    Ctr4x32 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return ((uint64_t)r.v[0] << 32) | r.v[1];
}

// ------------------------------------------------------------- small vectors
static inline double dot3(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }
static inline void cross3(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// ------------------------------------------------------------------ geometry
struct Geom {
    int nn = 0, nc = 0, nf = 0, nbf = 0;
    std::vector<double> xyz;          // [3*nn] node-major (x,y,z per node)
    std::vector<int32_t> tet;         // [4*nc]
    std::vector<int32_t> tet_face;    // [4*nc] face opposite local node k
    std::vector<int8_t> tet_sign;     // [4*nc] +1 if the tet owns the face
    std::vector<int32_t> f_owner, f_nbr, f_owner_k, f_nbr_k, f_bc;
    std::vector<double> f_n, f_area, f_c, f_d, f_t1, f_t2;  // [3*nf] or [nf]
    std::vector<double> vol, cen, dS;                      // [nc], [3*nc], [3*nc]
};

static bool build_geometry(Geom& g, int nn, const double* xyz, int nc, const int32_t* tets,
                           int nbf, const int32_t* bf, const int32_t* btag, int n_bc, std::string& err) {
    g.nn = nn; g.nc = nc;
    g.xyz.assign(xyz, xyz + 3 * (size_t)nn);
    g.tet.assign(tets, tets + 4 * (size_t)nc);
    g.tet_face.assign(4 * (size_t)nc, -1);
    g.tet_sign.assign(4 * (size_t)nc, 0);
    g.vol.resize(nc); g.cen.resize(3 * (size_t)nc); g.dS.resize(3 * (size_t)nc);
    auto P = [&](int node) { return &g.xyz[3 * (size_t)node]; };
    for (int i = 0; i < nc; ++i) {
        for (int k = 0; k < 4; ++k) {
            int v = g.tet[4 * i + k];
            if (v < 0 || v >= nn) { err = "tet node index out of range"; return false; }
        }
        const double *p0 = P(g.tet[4 * i]), *p1 = P(g.tet[4 * i + 1]), *p2 = P(g.tet[4 * i + 2]), *p3 = P(g.tet[4 * i + 3]);
        double a[3], b[3], c[3], bxc[3];
        for (int d = 0; d < 3; ++d) { a[d] = p1[d] - p0[d]; b[d] = p2[d] - p0[d]; c[d] = p3[d] - p0[d]; }
        cross3(b, c, bxc);
        double V = dot3(a, bxc) / 6.0;
        if (!(V > 0.0)) { err = "tet " + std::to_string(i) + " has non-positive volume"; return false; }
        g.vol[i] = V;
        for (int d = 0; d < 3; ++d) g.cen[3 * i + d] = (((p0[d] + p1[d]) + p2[d]) + p3[d]) * 0.25;
    }
    // Face matching on sorted node triples; faces numbered by first appearance.
    std::map<std::array<int, 3>, int> fmap;
    for (int i = 0; i < nc; ++i) {
        for (int k = 0; k < 4; ++k) {
            std::array<int, 3> key;
            int j = 0;
            for (int l = 0; l < 4; ++l) if (l != k) key[j++] = g.tet[4 * i + l];
            std::sort(key.begin(), key.end());
            auto it = fmap.find(key);
            if (it == fmap.end()) {
                int f = (int)g.f_owner.size();
                fmap[key] = f;
                g.f_owner.push_back(i); g.f_owner_k.push_back(k);
                g.f_nbr.push_back(-1); g.f_nbr_k.push_back(-1);
                g.tet_face[4 * i + k] = f; g.tet_sign[4 * i + k] = 1;
            } else {
                int f = it->second;
                if (g.f_nbr[f] >= 0) { err = "face shared by more than two tets"; return false; }
                g.f_nbr[f] = i; g.f_nbr_k[f] = k;
                g.tet_face[4 * i + k] = f; g.tet_sign[4 * i + k] = -1;
            }
        }
    }
    int nf = (int)g.f_owner.size();
    g.nf = nf;
    g.f_bc.assign(nf, -1);
    for (int b = 0; b < nbf; ++b) {
        std::array<int, 3> key = {bf[3 * b], bf[3 * b + 1], bf[3 * b + 2]};
        std::sort(key.begin(), key.end());
        auto it = fmap.find(key);
        if (it == fmap.end()) { err = "boundary face " + std::to_string(b) + " is not a tet face"; return false; }
        int f = it->second;
        if (g.f_nbr[f] >= 0) { err = "boundary face " + std::to_string(b) + " is interior"; return false; }
        if (btag[b] < 0 || btag[b] >= n_bc) { err = "boundary tag out of range"; return false; }
        if (g.f_bc[f] >= 0) { err = "boundary face listed twice"; return false; }
        g.f_bc[f] = btag[b];
    }
    g.nbf = 0;
    for (int f = 0; f < nf; ++f) {
        if (g.f_nbr[f] < 0) {
            if (g.f_bc[f] < 0) { err = "unmatched face " + std::to_string(f) + " has no boundary tag"; return false; }
            g.nbf++;
        }
    }
    // Face geometry: normal from the cross product of the sorted triple, turned
    // to point out of the owner; centroid; plane offset d = n . centroid.
    g.f_n.resize(3 * (size_t)nf); g.f_area.resize(nf); g.f_c.resize(3 * (size_t)nf); g.f_d.resize(nf);
    g.f_t1.resize(3 * (size_t)nf); g.f_t2.resize(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f) {
        int o = g.f_owner[f], k = g.f_owner_k[f];
        int tri[3], j = 0;
        for (int l = 0; l < 4; ++l) if (l != k) tri[j++] = g.tet[4 * o + l];
        std::sort(tri, tri + 3);
        const double *pa = P(tri[0]), *pb = P(tri[1]), *pc = P(tri[2]), *po = P(g.tet[4 * o + k]);
        double e1[3], e2[3], N[3], w[3];
        for (int d = 0; d < 3; ++d) { e1[d] = pb[d] - pa[d]; e2[d] = pc[d] - pa[d]; w[d] = po[d] - pa[d]; }
        cross3(e1, e2, N);
        double s = dot3(N, w);
        if (s == 0.0) { err = "degenerate face"; return false; }
        if (s > 0.0) { N[0] = -N[0]; N[1] = -N[1]; N[2] = -N[2]; }
        double len = std::sqrt(dot3(N, N));
        double* n = &g.f_n[3 * (size_t)f];
        for (int d = 0; d < 3; ++d) n[d] = N[d] / len;
        g.f_area[f] = 0.5 * len;
        double* c = &g.f_c[3 * (size_t)f];
        for (int d = 0; d < 3; ++d) c[d] = ((pa[d] + pb[d]) + pc[d]) / 3.0;
        g.f_d[f] = dot3(n, c);
        // Tangent basis: t1 = (e_a x n)/|e_a x n| with a the axis of smallest |n_a|.
        int a = 0;
        for (int d = 1; d < 3; ++d) if (std::fabs(n[d]) < std::fabs(n[a])) a = d;
        double ea[3] = {0.0, 0.0, 0.0}; ea[a] = 1.0;
        double t1[3], t2[3];
        cross3(ea, n, t1);
        double l1 = std::sqrt(dot3(t1, t1));
        for (int d = 0; d < 3; ++d) t1[d] = t1[d] / l1;
        cross3(n, t1, t2);
        for (int d = 0; d < 3; ++d) { g.f_t1[3 * (size_t)f + d] = t1[d]; g.f_t2[3 * (size_t)f + d] = t2[d]; }
    }
    // Projected areas (Sec. 2.4 (a)): dS^x = 1/2 sum_j |S^x_ij| with S = |S| n.
    for (int i = 0; i < nc; ++i) {
        for (int d = 0; d < 3; ++d) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) {
                int f = g.tet_face[4 * i + k];
                acc = acc + std::fabs(g.f_n[3 * (size_t)f + d] * g.f_area[f]);
            }
            g.dS[3 * i + d] = 0.5 * acc;
        }
    }
    return true;
}

// ------------------------------------------------------------- primitives
// Sec. 2: W = (rho, rho U, rho E), rho E = 1/2 rho |U|^2 + (3+K)/2 p with K
// internal degrees of freedom, p = rho R T, lambda = 1/(2RT).
struct Prim { double rho, U[3], p, T, lam; };
static inline Prim prim_of(const double* W, double R, int K) {
    Prim s;
    s.rho = W[0];
    for (int d = 0; d < 3; ++d) s.U[d] = W[1 + d] / s.rho;
    double U2 = (s.U[0] * s.U[0] + s.U[1] * s.U[1]) + s.U[2] * s.U[2];
    s.p = (W[4] - 0.5 * (s.rho * U2)) / (1.5 + 0.5 * (double)K);
    s.T = s.p / (s.rho * R);
    s.lam = s.rho / (2.0 * s.p);
    return s;
}

// tau = mu_ref / p (T / T_ref)^omega  (Eq. tau_via_T_ref), with the power written
// as exp(omega log(T/T_ref)) through the bit-reproducible exp_d/log_d.
static inline double tau_cell(const Prim& s, const orc_params& P) {
    return (P.mu_ref / s.p) * exp_d(P.omega * log_d(s.T / P.T_ref));
}

// ------------------------------------------------------- time coefficients
// q1..q5 = int_0^dt c1..c5 dt (Sec. 2.1) and the free-transport coefficients of
// the collisional wave (Sec. 2.3): a4 = q4 - dt e^{-dt/tau}, a5 = q5 + dt^2/2 e^{-dt/tau}.
// For x = dt/tau < 1 each is tau^p times a power series in x whose k-th
// coefficient follows from expanding e^{-x}; otherwise the closed forms are used.
static void qcoef(double dt, double tau, double q[7]) {
    double x = dt / tau;
    if (x < 1.0) {
        double s[7] = {0, 0, 0, 0, 0, 0, 0};
        double term = 1.0;  // x^k / k!
        for (int k = 1; k <= 30; ++k) {
            term = term * x / (double)k;
            double sg = (k % 2 == 0) ? 1.0 : -1.0;  // (-1)^k
            if (k >= 2) s[0] += sg * term;                                   // q1/tau
            if (k >= 3) s[1] += -sg * (double)(2 - k) * term;                // q2/tau^2
            if (k >= 3) s[2] += -sg * term;                                  // q3/tau^2
            s[3] += -sg * term;                                              // q4/tau
            if (k >= 2) s[4] += -sg * (double)(k - 1) * term;                // q5/tau^2
            if (k >= 2) s[5] += -sg * (double)(1 - k) * term;                // a4/tau
            if (k >= 3) s[6] += sg * 0.5 * (double)((k - 1) * (k - 2)) * term;  // a5/tau^2
        }
        double t2 = tau * tau;
        q[0] = tau * s[0]; q[1] = t2 * s[1]; q[2] = t2 * s[2]; q[3] = tau * s[3];
        q[4] = t2 * s[4]; q[5] = tau * s[5]; q[6] = t2 * s[6];
    } else {
        double e = std::exp(-x);
        double ph = -std::expm1(-x);  // 1 - e^{-x}
        q[0] = dt - tau * ph;
        q[1] = 2.0 * tau * tau * ph - tau * dt - tau * dt * e;
        q[2] = 0.5 * dt * dt - tau * dt + tau * tau * ph;
        q[3] = tau * ph;
        q[4] = tau * dt * e - tau * tau * ph;
        q[5] = q[3] - dt * e;
        q[6] = q[4] + 0.5 * dt * dt * e;
    }
}

// ------------------------------------------------------ Maxwellian moments
// Moments <u_n^k>, k = 0..4, of the normalised 1D Maxwellian in the normal
// direction over u_n > 0 (half = +1), u_n < 0 (half = -1) or all u_n (half = 0),
// by the recurrence <u^{k+2}> = Un <u^{k+1}> + (k+1)/(2 lambda) <u^k>.
static void un_moments(double Un, double lam, int half, double M[5]) {
    if (half == 0) {
        M[0] = 1.0; M[1] = Un;
    } else {
        double a = std::sqrt(lam) * Un;
        double edge = 0.5 * std::exp(-lam * Un * Un) / std::sqrt(PI * lam);
        if (half > 0) { M[0] = 0.5 * std::erfc(-a); M[1] = Un * M[0] + edge; }
        else          { M[0] = 0.5 * std::erfc(a);  M[1] = Un * M[0] - edge; }
    }
    for (int k = 0; k < 3; ++k) M[k + 2] = Un * M[k + 1] + (double)(k + 1) / (2.0 * lam) * M[k];
}

// H = int g psi du dxi and G = int u_n g psi du dxi over the half space, for a
// unit-density Maxwellian with velocity U = Un n + Ut and lambda;
// psi = (1, u, (|u|^2 + |xi|^2)/2) with K internal degrees of freedom xi.
static void half_moments(double Un, const double* Ut, const double* n, double lam, int half, int K,
                         double H[5], double G[5]) {
    double M[5];
    un_moments(Un, lam, half, M);
    double Ut2 = (Ut[0] * Ut[0] + Ut[1] * Ut[1]) + Ut[2] * Ut[2];
    // <|u_t|^2> of the two tangential directions, then + <|xi|^2> = K/(2 lambda)
    double tv = (Ut2 + 1.0 / lam) + (double)K * (0.5 / lam);
    H[0] = M[0];
    G[0] = M[1];
    for (int d = 0; d < 3; ++d) {
        H[1 + d] = M[1] * n[d] + M[0] * Ut[d];
        G[1 + d] = M[2] * n[d] + M[1] * Ut[d];
    }
    H[4] = 0.5 * (M[2] + M[0] * tv);
    G[4] = 0.5 * (M[3] + M[1] * tv);
}

struct FaceState { double rho, rhoh, Un, Ut[3], lam, p, T; };
static FaceState face_state(const double* W, double rhoh, const double* n, double R, int K) {
    Prim s = prim_of(W, R, K);
    FaceState f;
    f.rho = s.rho; f.rhoh = rhoh; f.lam = s.lam; f.p = s.p; f.T = s.T;
    f.Un = dot3(s.U, n);
    for (int d = 0; d < 3; ++d) f.Ut[d] = s.U[d] - f.Un * n[d];
    return f;
}

// ---------------------------------------------------------------- face flux
// Time-integrated flux per unit area through a face with unit normal n (L -> R):
//   F = F^eq + F^{fr,wave}
//   F^eq       = int u.n (q1 g0) psi du                    (Eq. macroscopic fluxes,
//                first order: g_x = g_t = 0)
//   F^{fr,wave}= int u.n [(q4 - dt e^{-dt/tau}) g0^h] psi du   (Sec. 2.3, g_x^h = 0)
// with W0 = int_{u.n>0} g_L psi + int_{u.n<0} g_R psi (compatibility condition,
// Sec. 2.1) and reading: g0^h is the upwind hydrodynamic Maxwellian
// (rho^h_L/rho_L) g_L for u.n >= 0 and (rho^h_R/rho_R) g_R for u.n < 0.
// Face relaxation time (Sec. 2.4 (d)): tau = mu(T0)/p0 + C2 |pL-pR|/|pL+pR| dt.
// ghost_hydro: the R side is a far-field ghost that emits no particles, so its
// incoming half carries the full UGKS free-transport coefficient q4.
// gks: a step without particles (the gas-kinetic scheme the method reduces to
// when no particle is sampled, Sec. 3.2): both halves carry q4.
static void interior_flux(const FaceState& L, const FaceState& Rs, bool ghost_hydro, bool gks,
                          const double* n, double dt, const orc_params& P, double F[5]) {
    double HL[5], GL[5], HR[5], GR[5];
    half_moments(L.Un, L.Ut, n, L.lam, +1, P.K, HL, GL);
    half_moments(Rs.Un, Rs.Ut, n, Rs.lam, -1, P.K, HR, GR);
    double W0[5];
    for (int q = 0; q < 5; ++q) W0[q] = L.rho * HL[q] + Rs.rho * HR[q];
    Prim s0 = prim_of(W0, P.R, P.K);
    double tau = P.mu_ref * std::pow(s0.T / P.T_ref, P.omega) / s0.p
               + P.C2 * std::fabs(L.p - Rs.p) / std::fabs(L.p + Rs.p) * dt;
    double q[7];
    qcoef(dt, tau, q);
    double Un0 = dot3(s0.U, n), Ut0[3];
    for (int d = 0; d < 3; ++d) Ut0[d] = s0.U[d] - Un0 * n[d];
    double H0[5], G0[5];
    half_moments(Un0, Ut0, n, s0.lam, 0, P.K, H0, G0);
    double cL = gks ? q[3] : q[5];
    double cR = (ghost_hydro || gks) ? q[3] : q[5];
    for (int k = 0; k < 5; ++k)
        F[k] = q[0] * (s0.rho * G0[k]) + cL * (L.rhoh * GL[k]) + cR * (Rs.rhoh * GR[k]);
}

// Diffuse isothermal wall (Sec. 2.4 (e)), n pointing from the gas into the wall.
// Incoming half: the interior state as g0 and f0 with the cell's tau; emitted
// half: the wall Maxwellian g_w(T_w, U_w) over the whole step with rho_w from
// zero net mass flux of the wave (reading: particles reflect individually).
static void wall_flux(const FaceState& L, double tau, const orc_bc& bc, const double* n,
                      double dt, bool gks, const orc_params& P, double F[5]) {
    double q[7];
    qcoef(dt, tau, q);
    double HL[5], GL[5];
    half_moments(L.Un, L.Ut, n, L.lam, +1, P.K, HL, GL);
    double Gin[5];
    const double c4 = gks ? q[3] : q[5];
    for (int k = 0; k < 5; ++k) Gin[k] = q[0] * (L.rho * GL[k]) + c4 * (L.rhoh * GL[k]);
    double lamw = 1.0 / (2.0 * P.R * bc.T_w);
    double Uwn = dot3(bc.U_w, n), Uwt[3];
    for (int d = 0; d < 3; ++d) Uwt[d] = bc.U_w[d] - Uwn * n[d];
    double Hw[5], Gw[5];
    half_moments(Uwn, Uwt, n, lamw, -1, P.K, Hw, Gw);
    double rhow = -Gin[0] / (dt * Gw[0]);
    for (int k = 0; k < 5; ++k) F[k] = Gin[k] + dt * rhow * Gw[k];
}

static void boundary_flux(const double* WL, double rhohL, double tauL, const orc_bc& bc,
                          const double* n, double dt, bool gks, const orc_params& P, double F[5]) {
    FaceState L = face_state(WL, rhohL, n, P.R, P.K);
    if (bc.type == ORC_BC_DIFFUSE_WALL) { wall_flux(L, tauL, bc, n, dt, gks, P, F); return; }
    if (bc.type == ORC_BC_SPECULAR) {
        // Mirror ghost: same state with the normal velocity reversed.  Only the
        // normal momentum flux survives; mass, energy and shear are zero.
        FaceState Rg = L; Rg.Un = -L.Un;
        double Ff[5];
        interior_flux(L, Rg, false, gks, n, dt, P, Ff);
        double fn = dot3(&Ff[1], n);
        F[0] = 0.0; F[4] = 0.0;
        for (int d = 0; d < 3; ++d) F[1 + d] = fn * n[d];
        return;
    }
    // Far field: inflow ghost = prescribed state, outflow ghost = interior state;
    // both all-hydrodynamic and emitting no particles (reading).
    FaceState Rg = (bc.type == ORC_BC_INFLOW) ? face_state(bc.W_in, bc.W_in[0], n, P.R, P.K) : L;
    Rg.rhoh = Rg.rho;
    interior_flux(L, Rg, true, gks, n, dt, P, F);
}

// ------------------------------------------------ second-order reconstruction
// Least-squares gradients with Venkatakrishnan's limiter (Sec. 2.1).  Readings:
// inverse-distance-squared weights over the 4 face neighbours; at boundary faces
// a ghost at the mirror image of the centroid across the face holding the
// ghost state (specular: mirrored velocity; far field: W_in, all hydro; wall
// and outflow: the cell's own value); epsilon^2 = (K h)^3, h = |Omega|^(1/3).

// Ghost conservative state and rho^h across boundary face with outward n.
static void ghost_state(const double* Wi, double rhohi, const orc_bc& bc, const double* n, double* Wg, double* rhohg) {
    for (int q = 0; q < 5; ++q) Wg[q] = Wi[q];
    *rhohg = rhohi;
    if (bc.type == ORC_BC_SPECULAR) {
        double mn = dot3(&Wi[1], n);
        for (int d = 0; d < 3; ++d) Wg[1 + d] = Wi[1 + d] - 2.0 * mn * n[d];
    } else if (bc.type == ORC_BC_INFLOW) {
        for (int q = 0; q < 5; ++q) Wg[q] = bc.W_in[q];
        *rhohg = bc.W_in[0];
    }
}

// Venkatakrishnan's limiter function for an extrapolated difference d2 and the
// allowed difference d1 (same sign), with epsilon^2 = eps2.
static double venkat(double d1, double d2, double eps2) {
    double num = (d1 * d1 + eps2) * d2 + 2.0 * d2 * d2 * d1;
    double den = d2 * (d1 * d1 + 2.0 * d2 * d2 + d1 * d2 + eps2);
    return num / den;
}

// Limited gradients of W (5 x 3, row-major [q][d]) and rho^h (3) of every cell.
// phi_io (optional, [6][nc]): with phi_given the limiter values are taken from
// it instead of computed (a frozen limiter); otherwise the computed ones are
// stored there.
static void limited_gradients(const Geom& g, const orc_params& P, const std::vector<double>& W,
                              const std::vector<double>& rhoh, bool limit,
                              std::vector<double>& gradW, std::vector<double>& gradH,
                              double* phi_io = nullptr, bool phi_given = false) {
    const int nc = g.nc;
    gradW.assign(15 * (size_t)nc, 0.0);
    gradH.assign(3 * (size_t)nc, 0.0);
    for (int i = 0; i < nc; ++i) {
        const double* xi = &g.cen[3 * (size_t)i];
        double Wi[5];
        for (int q = 0; q < 5; ++q) Wi[q] = W[(size_t)q * nc + i];
        // neighbour (or ghost) positions and values, 6 quantities: W[5], rho^h
        double dx[4][3], val[4][6], w[4];
        for (int k = 0; k < 4; ++k) {
            int f = g.tet_face[4 * i + k];
            int j = g.tet_sign[4 * i + k] > 0 ? g.f_nbr[f] : g.f_owner[f];
            if (j >= 0) {
                for (int d = 0; d < 3; ++d) dx[k][d] = g.cen[3 * (size_t)j + d] - xi[d];
                for (int q = 0; q < 5; ++q) val[k][q] = W[(size_t)q * nc + j];
                val[k][5] = rhoh[j];
            } else {
                const double* n = &g.f_n[3 * (size_t)f];
                const double* xf = &g.f_c[3 * (size_t)f];
                double h = (xf[0] - xi[0]) * n[0] + (xf[1] - xi[1]) * n[1] + (xf[2] - xi[2]) * n[2];
                for (int d = 0; d < 3; ++d) dx[k][d] = 2.0 * h * n[d];
                double Wg[5], hg;
                ghost_state(Wi, rhoh[i], P.bc[g.f_bc[f]], n, Wg, &hg);
                for (int q = 0; q < 5; ++q) val[k][q] = Wg[q];
                val[k][5] = hg;
            }
            w[k] = 1.0 / dot3(dx[k], dx[k]);
        }
        // normal equations A grad = b, A = sum w dx dx^T (3 x 3), solved by
        // Gaussian elimination with partial pivoting for each quantity
        double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int k = 0; k < 4; ++k)
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) A[r][c] += w[k] * dx[k][r] * dx[k][c];
        const double self[6] = {Wi[0], Wi[1], Wi[2], Wi[3], Wi[4], rhoh[i]};
        double grad[6][3];
        for (int q = 0; q < 6; ++q) {
            double M[3][4];
            for (int r = 0; r < 3; ++r) {
                for (int c = 0; c < 3; ++c) M[r][c] = A[r][c];
                double b = 0.0;
                for (int k = 0; k < 4; ++k) b += w[k] * dx[k][r] * (val[k][q] - self[q]);
                M[r][3] = b;
            }
            for (int c = 0; c < 3; ++c) {
                int piv = c;
                for (int r = c + 1; r < 3; ++r) if (std::fabs(M[r][c]) > std::fabs(M[piv][c])) piv = r;
                for (int cc = 0; cc < 4; ++cc) std::swap(M[c][cc], M[piv][cc]);
                for (int r = c + 1; r < 3; ++r) {
                    double fct = M[r][c] / M[c][c];
                    for (int cc = c; cc < 4; ++cc) M[r][cc] -= fct * M[c][cc];
                }
            }
            for (int r = 2; r >= 0; --r) {
                double acc = M[r][3];
                for (int c = r + 1; c < 3; ++c) acc -= M[r][c] * grad[q][c];
                grad[q][r] = acc / M[r][r];
            }
            double phi = 1.0;
            if (phi_given) {
                phi = phi_io[(size_t)q * nc + i];
            } else if (limit) {
                double vmax = self[q], vmin = self[q];
                for (int k = 0; k < 4; ++k) { vmax = std::max(vmax, val[k][q]); vmin = std::min(vmin, val[k][q]); }
                double h = std::cbrt(g.vol[i]);
                double eps2 = std::pow(P.venkat_K * h, 3.0);
                for (int k = 0; k < 4; ++k) {
                    int f = g.tet_face[4 * i + k];
                    const double* xf = &g.f_c[3 * (size_t)f];
                    double d2 = grad[q][0] * (xf[0] - xi[0]) + grad[q][1] * (xf[1] - xi[1]) + grad[q][2] * (xf[2] - xi[2]);
                    double pk = 1.0;
                    if (d2 > 0.0) pk = venkat(vmax - self[q], d2, eps2);
                    else if (d2 < 0.0) pk = venkat(vmin - self[q], d2, eps2);
                    phi = std::min(phi, pk);
                }
            }
            if (phi_io && !phi_given) phi_io[(size_t)q * nc + i] = phi;
            for (int d = 0; d < 3; ++d) {
                if (q < 5) gradW[15 * (size_t)i + 3 * q + d] = phi * grad[q][d];
                else gradH[3 * (size_t)i + d] = phi * grad[q][d];
            }
        }
    }
}

// ---- velocity moments of a unit-density Maxwellian in the face frame
// (u along n, v along t1, w along t2), by explicit expansion over monomials.
// a monomial c u^a v^b w^e |xi|^(2x) (xi: the K internal degrees of freedom)
struct Term { double c; int a, b, e, x; };
typedef std::vector<Term> Poly;

// 1D moments of the frame directions and <|xi|^(2j)>, j = 0..3
struct FrameMom { double n[8], t1[8], t2[8], xi[4]; };

// <u^k>, k = 0..7, of the normalised 1D Maxwellian (mean m, lambda), over all u
// (half = 0) or the half line u > 0 (+1) / u < 0 (-1).
static void moments1d(double m, double lam, int half, double* M) {
    if (half == 0) { M[0] = 1.0; M[1] = m; }
    else {
        double a = std::sqrt(lam) * m;
        double edge = 0.5 * std::exp(-lam * m * m) / std::sqrt(PI * lam);
        if (half > 0) { M[0] = 0.5 * std::erfc(-a); M[1] = m * M[0] + edge; }
        else          { M[0] = 0.5 * std::erfc(a);  M[1] = m * M[0] - edge; }
    }
    for (int k = 0; k < 6; ++k) M[k + 2] = m * M[k + 1] + (double)(k + 1) / (2.0 * lam) * M[k];
}

static FrameMom frame_moments(const double* Uf, double lam, int half, int K) {
    FrameMom F;
    moments1d(Uf[0], lam, half, F.n);
    moments1d(Uf[1], lam, 0, F.t1);
    moments1d(Uf[2], lam, 0, F.t2);
    // |xi|^2 is a sum of K squared normals of variance 1/(2 lambda):
    // <|xi|^(2j)> = K (K+2) ... (K+2j-2) / (2 lambda)^j
    F.xi[0] = 1.0;
    for (int j = 1; j < 4; ++j) F.xi[j] = F.xi[j - 1] * (double)(K + 2 * (j - 1)) / (2.0 * lam);
    return F;
}

static double expect(const FrameMom& M, const Poly& P) {
    double s = 0.0;
    for (const Term& t : P) s += t.c * M.n[t.a] * M.t1[t.b] * M.t2[t.e] * M.xi[t.x];
    return s;
}

static Poly mul(const Poly& A, const Poly& B) {
    Poly C;
    for (const Term& x : A)
        for (const Term& y : B) C.push_back(Term{x.c * y.c, x.a + y.a, x.b + y.b, x.e + y.e, x.x + y.x});
    return C;
}

// psi_k in the face frame: 1, u, v, w, (u^2 + v^2 + w^2 + |xi|^2)/2
static Poly psi(int k) {
    switch (k) {
        case 0: return Poly{{1.0, 0, 0, 0, 0}};
        case 1: return Poly{{1.0, 1, 0, 0, 0}};
        case 2: return Poly{{1.0, 0, 1, 0, 0}};
        case 3: return Poly{{1.0, 0, 0, 1, 0}};
        default: return Poly{{0.5, 2, 0, 0, 0}, {0.5, 0, 2, 0, 0}, {0.5, 0, 0, 2, 0}, {0.5, 0, 0, 0, 1}};
    }
}
static Poly lin(const double* a) {  // a . psi
    return Poly{{a[0], 0, 0, 0, 0}, {a[1], 1, 0, 0, 0}, {a[2], 0, 1, 0, 0}, {a[3], 0, 0, 1, 0},
                {0.5 * a[4], 2, 0, 0, 0}, {0.5 * a[4], 0, 2, 0, 0}, {0.5 * a[4], 0, 0, 2, 0},
                {0.5 * a[4], 0, 0, 0, 1}};
}
static Poly coord(int d) { return Poly{{1.0, d == 0 ? 1 : 0, d == 1 ? 1 : 0, d == 2 ? 1 : 0, 0}}; }

// Micro slope a with <psi psi^T> a = b for the unit Maxwellian (Uf, lam):
// the moment matrix built from moments, solved by Gaussian elimination.
static void micro_slope(const double* Uf, double lam, int K, const double* b, double* a) {
    FrameMom M = frame_moments(Uf, lam, 0, K);
    double A[5][6];
    for (int r = 0; r < 5; ++r) {
        for (int c = 0; c < 5; ++c) A[r][c] = expect(M, mul(psi(r), psi(c)));
        A[r][5] = b[r];
    }
    for (int c = 0; c < 5; ++c) {
        int piv = c;
        for (int r = c + 1; r < 5; ++r) if (std::fabs(A[r][c]) > std::fabs(A[piv][c])) piv = r;
        for (int cc = 0; cc < 6; ++cc) std::swap(A[c][cc], A[piv][cc]);
        for (int r = c + 1; r < 5; ++r) {
            double f = A[r][c] / A[c][c];
            for (int cc = c; cc < 6; ++cc) A[r][cc] -= f * A[c][cc];
        }
    }
    for (int r = 4; r >= 0; --r) {
        double acc = A[r][5];
        for (int c = r + 1; c < 5; ++c) acc -= A[r][c] * a[c];
        a[r] = acc / A[r][r];
    }
}

// Face frame of a face: rows n, t1, t2.
struct Frame { double r[3][3]; };
static void to_frame(const Frame& R, const double* v, double* out) {
    for (int i = 0; i < 3; ++i) out[i] = dot3(R.r[i], v);
}
// W (lab) -> W (frame): rotate the momentum components.
static void state_to_frame(const Frame& R, const double* W, double* Wf) {
    Wf[0] = W[0]; to_frame(R, &W[1], &Wf[1]); Wf[4] = W[4];
}
// gradient [q][d] (lab) -> slopes along the frame directions, momentum rotated:
// out[dd][q] = d/d(frame dir dd) of the frame-rotated W_q.
static void grad_to_frame(const Frame& R, const double* gW, double out[3][5]) {
    for (int dd = 0; dd < 3; ++dd) {
        double g[5];
        for (int q = 0; q < 5; ++q) g[q] = dot3(&gW[3 * q], R.r[dd]);  // directional derivative
        out[dd][0] = g[0];
        double m[3] = {g[1], g[2], g[3]};
        to_frame(R, m, &out[dd][1]);
        out[dd][4] = g[4];
    }
}

static Frame frame_of(const double* n) {
    Frame R;
    int a = 0;
    for (int d = 1; d < 3; ++d) if (std::fabs(n[d]) < std::fabs(n[a])) a = d;
    double ea[3] = {0.0, 0.0, 0.0}; ea[a] = 1.0;
    double t1[3], t2[3];
    cross3(ea, n, t1);
    double l1 = std::sqrt(dot3(t1, t1));
    for (int d = 0; d < 3; ++d) t1[d] = t1[d] / l1;
    cross3(n, t1, t2);
    for (int d = 0; d < 3; ++d) { R.r[0][d] = n[d]; R.r[1][d] = t1[d]; R.r[2][d] = t2[d]; }
    return R;
}

static void frame_to_lab(const Frame& R, const double* Ff, double* F) {
    F[0] = Ff[0];
    for (int d = 0; d < 3; ++d) F[1 + d] = (Ff[1] * R.r[0][d] + Ff[2] * R.r[1][d]) + Ff[3] * R.r[2][d];
    F[4] = Ff[4];
}

struct SideO2 {
    double W[5];   // frame state at the face
    double rhoh;
    double U[3], lam;
    double dW[3][5];   // frame slopes of W along n, t1, t2
    double dWh[3][5];  // frame slopes of W^h = (rho^h/rho) W
};

static bool side_o2(const Frame& R, const double* Wlab, double rhoh, const double* gW, const double* gH,
                    const double* dx, int K, SideO2& S) {
    // reconstruct W and rho^h at the face from the cell values and limited gradients
    double Wface[5];
    for (int q = 0; q < 5; ++q) Wface[q] = Wlab[q] + dot3(&gW[3 * q], dx);
    double rh = rhoh + dot3(gH, dx);
    Prim pr = prim_of(Wface, 1.0, K);
    if (!(Wface[0] > 0.0) || !(pr.p > 0.0)) return false;
    state_to_frame(R, Wface, S.W);
    S.rhoh = rh;
    for (int d = 0; d < 3; ++d) S.U[d] = S.W[1 + d] / S.W[0];
    S.lam = pr.lam;
    grad_to_frame(R, gW, S.dW);
    // grad of (rho^h/rho) W = (rho^h/rho) grad W + W grad(rho^h/rho),
    // grad(rho^h/rho) = (grad rho^h - (rho^h/rho) grad rho) / rho
    double ratio = rh / S.W[0];
    double gr[3];
    for (int d = 0; d < 3; ++d) gr[d] = (dot3(gH, R.r[d]) - ratio * S.dW[d][0]) / S.W[0];
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 5; ++q) S.dWh[d][q] = ratio * S.dW[d][q] + S.W[q] * gr[d];
    return true;
}

static SideO2 side_o1(const Frame& R, const double* Wlab, double rhoh, int K) {
    SideO2 S;
    state_to_frame(R, Wlab, S.W);
    S.rhoh = rhoh;
    Prim pr = prim_of(Wlab, 1.0, K);
    for (int d = 0; d < 3; ++d) S.U[d] = S.W[1 + d] / S.W[0];
    S.lam = pr.lam;
    for (int d = 0; d < 3; ++d) for (int q = 0; q < 5; ++q) { S.dW[d][q] = 0.0; S.dWh[d][q] = 0.0; }
    return S;
}

// Second-order flux through an interior face (Sec. 2.1, 2.3), in the face frame:
//   F^eq       = int u_n [q1 g0 + q2 u.g_x + q3 g_t] psi
//   F^{fr,wave}= int u_n [a4 g0^h + a5 u.g_x^h] psi  (upwind: L for u_n > 0, R for u_n < 0)
// with g_x from W_x = (grad W_L + grad W_R)/2 (reading), g_t from
// W_t = -int u.g_x psi, and all slopes solved from the moment system.
static void interior_flux_o2(const SideO2& L, const SideO2& Rs, const double* pLR, double dt, bool gks,
                             const orc_params& P, double Ff[5]) {
    FrameMom ML = frame_moments(L.U, L.lam, +1, P.K), MR = frame_moments(Rs.U, Rs.lam, -1, P.K);
    double W0[5];
    for (int k = 0; k < 5; ++k) W0[k] = L.W[0] * expect(ML, psi(k)) + Rs.W[0] * expect(MR, psi(k));
    Prim s0 = prim_of(W0, P.R, P.K);  // frame velocity components in s0.U
    double tau = P.mu_ref * std::pow(s0.T / P.T_ref, P.omega) / s0.p
               + P.C2 * std::fabs(pLR[0] - pLR[1]) / std::fabs(pLR[0] + pLR[1]) * dt;
    double q[7];
    qcoef(dt, tau, q);
    FrameMom M0 = frame_moments(s0.U, s0.lam, 0, P.K);
    // equilibrium slopes (with the density factor): a_d = M^-1 W_x,d
    double a0[3][5];
    for (int d = 0; d < 3; ++d) {
        double b[5];
        for (int k = 0; k < 5; ++k) b[k] = 0.5 * (L.dW[d][k] + Rs.dW[d][k]);
        micro_slope(s0.U, s0.lam, P.K, b, a0[d]);
    }
    double Wt[5], At[5];
    for (int k = 0; k < 5; ++k) {
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) acc += expect(M0, mul(mul(coord(d), lin(a0[d])), psi(k)));
        Wt[k] = -acc;
    }
    micro_slope(s0.U, s0.lam, P.K, Wt, At);
    // upwind hydrodynamic slopes a^h_d = M_side^-1 grad_d W^h
    double aL[3][5], aR[3][5];
    for (int d = 0; d < 3; ++d) {
        micro_slope(L.U, L.lam, P.K, L.dWh[d], aL[d]);
        micro_slope(Rs.U, Rs.lam, P.K, Rs.dWh[d], aR[d]);
    }
    const Poly un = coord(0);
    for (int k = 0; k < 5; ++k) {
        Poly unpsi = mul(un, psi(k));
        double feq = q[0] * s0.rho * expect(M0, unpsi) + q[2] * expect(M0, mul(unpsi, lin(At)));
        for (int d = 0; d < 3; ++d) feq += q[1] * expect(M0, mul(mul(unpsi, coord(d)), lin(a0[d])));
        // without particles (gks) the whole free transport q4, q5 is the wave's
        const double c4 = gks ? q[3] : q[5], c5 = gks ? q[4] : q[6];
        double ffr = c4 * (L.rhoh * expect(ML, unpsi) + Rs.rhoh * expect(MR, unpsi));
        for (int d = 0; d < 3; ++d) {
            Poly ud = mul(unpsi, coord(d));
            ffr += c5 * (expect(ML, mul(ud, lin(aL[d]))) + expect(MR, mul(ud, lin(aR[d]))));
        }
        Ff[k] = feq + ffr;
    }
    // Prandtl-number fix of the equilibrium part (reading, after the GKS
    // correction of Xu 2001): the energy flux gains (1/Pr - 1) q_n, q_n the
    // heat flux int (u_n - U0_n) |u - U0|^2/2 f_eq of the time-integrated
    // equilibrium part f_eq = q1 g0 + q2 u.g_x + q3 g_t, relative to U0.
    if (P.Pr > 0.0 && P.Pr != 1.0) {
        Poly sq;
        for (int d = 0; d < 3; ++d) {
            Poly rd = coord(d);
            rd.push_back(Term{-s0.U[d], 0, 0, 0});
            for (const Term& t : mul(rd, rd)) sq.push_back(Term{0.5 * t.c, t.a, t.b, t.e});
        }
        Poly rn = coord(0);
        rn.push_back(Term{-s0.U[0], 0, 0, 0});
        sq.push_back(Term{0.5, 0, 0, 0, 1});  // + |xi|^2 / 2
        const Poly h = mul(rn, sq);
        double qn = q[0] * s0.rho * expect(M0, h) + q[2] * expect(M0, mul(h, lin(At)));
        for (int d = 0; d < 3; ++d) qn += q[1] * expect(M0, mul(mul(h, coord(d)), lin(a0[d])));
        Ff[4] += (1.0 / P.Pr - 1.0) * qn;
    }
}

// One interior face at second order: reconstruct both sides (first order on a
// side whose reconstruction is not positive) and evaluate the O2 flux.
static void face_flux_o2(const Frame& R, const double* WL, double rhohL, const double* gWL, const double* gHL,
                         const double* dxL, const double* WR, double rhohR, const double* gWR,
                         const double* gHR, const double* dxR, double dt, bool gks, const orc_params& P,
                         double F[5]) {
    SideO2 L, Rs;
    if (!side_o2(R, WL, rhohL, gWL, gHL, dxL, P.K, L)) L = side_o1(R, WL, rhohL, P.K);
    if (!side_o2(R, WR, rhohR, gWR, gHR, dxR, P.K, Rs)) Rs = side_o1(R, WR, rhohR, P.K);
    double pLR[2] = {0.5 * L.W[0] / L.lam, 0.5 * Rs.W[0] / Rs.lam};
    double Ff[5];
    interior_flux_o2(L, Rs, pLR, dt, gks, P, Ff);
    frame_to_lab(R, Ff, F);
}

// ------------------------------------------------ first-order g_p sampling
// Option (sampling = 2): the hydrodynamic particles are drawn from the
// first-order g_p of Sec. 2.2 instead of the Maxwellian.  Reading: at the
// start of a step the collisional part represents the end of an interval of
// length dt, whose equilibrium, expanded about the cell's current state and
// averaged with the weights e^{-(t-t')/tau}/tau, is
//   g_p = g - c (u.grad g + g_t),  c = tau - dt e^{-dt/tau} / (1 - e^{-dt/tau})
// (the printed g_p with g0 moved to the end of the interval; c -> tau as
// tau/dt -> 0, the Chapman-Enskog distribution, and c -> dt/2 as tau/dt -> oo).
// grad g from the cell's limited least-squares gradient, g_t from
// W_t = -int u.grad g psi; both as (slope . psi) g.  With u = U + sqrt(RT) X,
// g_p / rho = N(X) (1 + phi(X)), phi = a0 + L.X + X^T Q X + (C.X)|X|^2, which
// is drawn by acceptance-rejection with the bound M = 1 + Phi,
// Phi = |a0| + 5|L| + 25|Q|_F + 125|C| (phi over |X| <= 5); where Phi > 1 the
// correction is scaled down to Phi = 1 (a limiter on the non-equilibrium part).
// Coefficients: [a0, L(3), Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, C(3), M].
static const int GP_NC = 14;
static const int GP_ATTEMPTS = 64;

static void gp_coefficients(const Prim& s, const double* gW, double tau, double dt, double R, double* out) {
    const double* U = s.U;
    const double sig = std::sqrt(R * s.T);
    // unit-density slopes: <psi psi^T> b_d = (d W / d x_d) / rho
    double b[3][5];
    for (int d = 0; d < 3; ++d) {
        double rhs[5];
        for (int q = 0; q < 5; ++q) rhs[q] = gW[3 * q + d] / s.rho;
        micro_slope(U, s.lam, 0, rhs, b[d]);
    }
    // W_t / rho = -sum_d <u_d psi (b_d . psi)>, <psi psi^T> B = W_t / rho
    FrameMom M0 = frame_moments(U, s.lam, 0, 0);
    double Wt[5], B[5];
    for (int k = 0; k < 5; ++k) {
        double acc = 0.0;
        for (int d = 0; d < 3; ++d) acc += expect(M0, mul(mul(coord(d), lin(b[d])), psi(k)));
        Wt[k] = -acc;
    }
    micro_slope(U, s.lam, 0, Wt, B);
    // P(u) = sum_d u_d (b_d . psi) + B . psi
    //      = B0 + v.u + u^T K u + (h/2)|u|^2 + (|u|^2/2)(beta.u)
    double v[3], K[3][3], beta[3];
    const double h = B[4];
    for (int j = 0; j < 3; ++j) {
        v[j] = B[1 + j] + b[j][0];
        beta[j] = b[j][4];
        for (int d = 0; d < 3; ++d) K[d][j] = b[d][1 + j];
    }
    const double UU = dot3(U, U), bU = dot3(beta, U);
    double KU[3];  // (K + K^T) U
    for (int d = 0; d < 3; ++d) {
        KU[d] = 0.0;
        for (int j = 0; j < 3; ++j) KU[d] += (K[d][j] + K[j][d]) * U[j];
    }
    double UKU = 0.0;
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < 3; ++j) UKU += U[d] * K[d][j] * U[j];
    double a0 = B[0] + dot3(v, U) + UKU + 0.5 * h * UU + 0.5 * UU * bU;
    double L[3], Q[3][3], C[3];
    for (int d = 0; d < 3; ++d) {
        L[d] = sig * (v[d] + KU[d] + h * U[d] + 0.5 * UU * beta[d] + bU * U[d]);
        C[d] = 0.5 * sig * sig * sig * beta[d];
        for (int j = 0; j < 3; ++j)
            Q[d][j] = sig * sig * (0.5 * (K[d][j] + K[j][d]) + 0.5 * (U[d] * beta[j] + U[j] * beta[d])
                                   + (d == j ? 0.5 * h + 0.5 * bU : 0.0));
    }
    const double e = exp_d(-(dt / tau));
    const double c = tau - dt * e / (1.0 - e);
    double co[13] = {a0, L[0], L[1], L[2], Q[0][0], Q[1][1], Q[2][2], Q[0][1], Q[0][2], Q[1][2], C[0], C[1], C[2]};
    for (int k = 0; k < 13; ++k) co[k] = -c * co[k];
    const double nL = std::sqrt(co[1] * co[1] + co[2] * co[2] + co[3] * co[3]);
    const double nQ = std::sqrt(co[4] * co[4] + co[5] * co[5] + co[6] * co[6]
                                + 2.0 * (co[7] * co[7] + co[8] * co[8] + co[9] * co[9]));
    const double nC = std::sqrt(co[10] * co[10] + co[11] * co[11] + co[12] * co[12]);
    double Phi = std::fabs(co[0]) + 5.0 * nL + 25.0 * nQ + 125.0 * nC;
    if (Phi > 1.0) {
        for (int k = 0; k < 13; ++k) co[k] = co[k] / Phi;
        Phi = 1.0;
    }
    for (int k = 0; k < 13; ++k) out[k] = co[k];
    out[13] = 1.0 + Phi;
}

// One acceptance-rejection draw of X ~ (1 + phi(X)) N(0, I) / (normalised)
// for particle `id` of a cell with coefficients c (first-order g_p), in the
// particle precision: attempt k draws three normals by Box-Muller from
// Philox counter (id, step, TAG_GP, 2k) and eta from (id, step, TAG_GP,
// 2k + 1), and accepts if eta M <= 1 + phi(X); after GP_ATTEMPTS attempts the
// last draw is kept.
template <class Real>
static void gp_draw(uint64_t seed, uint64_t step, const double* c, uint64_t id, double Xout[3]) {
    typedef Real R;
    const R a0 = (R)c[0], L0 = (R)c[1], L1 = (R)c[2], L2 = (R)c[3];
    const R Q0 = (R)c[4], Q1 = (R)c[5], Q2 = (R)c[6], Q3 = (R)c[7], Q4 = (R)c[8], Q5 = (R)c[9];
    const R C0 = (R)c[10], C1 = (R)c[11], C2 = (R)c[12], Mb = (R)c[13];
    R X[3] = {(R)0, (R)0, (R)0};
    for (int k = 0; k < GP_ATTEMPTS; ++k) {
        Ctr4 r = draw(seed, id, step, TAG_GP, (uint64_t)(2 * k));
        Ctr4 r2 = draw(seed, id, step, TAG_GP, (uint64_t)(2 * k + 1));
        R eta;
        if constexpr (std::is_same<Real, float>::value) {
            float sn, cs;
            float rad = std::sqrt(-2.0f * log_f(u01_f(r.v[0])));
            sincos2pi_f(u01_f(r.v[1]), &sn, &cs);
            X[0] = rad * cs; X[1] = rad * sn;
            rad = std::sqrt(-2.0f * log_f(u01_f(r.v[2])));
            sincos2pi_f(u01_f(r.v[3]), &sn, &cs);
            X[2] = rad * cs;
            eta = u01_f(r2.v[0]);
        } else {
            double sn, cs;
            double rad = std::sqrt(-2.0 * log_d(u01_d(r.v[0])));
            sincos2pi_d(u01_d(r.v[1]), &sn, &cs);
            X[0] = rad * cs; X[1] = rad * sn;
            rad = std::sqrt(-2.0 * log_d(u01_d(r.v[2])));
            sincos2pi_d(u01_d(r.v[3]), &sn, &cs);
            X[2] = rad * cs;
            eta = u01_d(r2.v[0]);
        }
        // phi = a0 + L.X + X^T Q X + (C.X) |X|^2, in this order
        const R lin = (L0 * X[0] + L1 * X[1]) + L2 * X[2];
        const R qd = ((Q0 * X[0]) * X[0] + (Q1 * X[1]) * X[1]) + (Q2 * X[2]) * X[2];
        const R qo = ((Q3 * X[0]) * X[1] + (Q4 * X[0]) * X[2]) + (Q5 * X[1]) * X[2];
        const R cub = ((C0 * X[0] + C1 * X[1]) + C2 * X[2]) * ((X[0] * X[0] + X[1] * X[1]) + X[2] * X[2]);
        const R phi = ((a0 + lin) + (qd + (qo + qo))) + cub;
        if (eta * Mb <= (R)1 + phi) break;
    }
    for (int d = 0; d < 3; ++d) Xout[d] = (double)X[d];
}

// ------------------------------------------------------------ particles
// e: internal energy per unit mass (|xi|^2, zero when K = 0), phi = m (1, u, (|u|^2 + e)/2)
template <class Real> struct Part { uint64_t id; int32_t cell; Real x[3]; Real u[3]; double m; Real e = (Real)0; };

// Internal energy of a particle with K internal degrees of freedom at spread
// sig = sqrt(RT): e = sum_{i<K} (sig N_i)^2, the normals N by Box-Muller from
// Philox counters (id, step, tag, idx0 + j), four per counter, summed in order
// in the particle precision.
template <class Real>
static Real internal_energy(uint64_t seed, uint64_t id, uint64_t step, uint64_t tag, uint64_t idx0, int K, Real sig) {
    Real e = (Real)0;
    for (int j = 0; 4 * j < K; ++j) {
        Ctr4 r = draw(seed, id, step, tag, idx0 + (uint64_t)j);
        Real N[4];
        if constexpr (std::is_same<Real, float>::value) {
            float sn, cs;
            float rad = std::sqrt(-2.0f * log_f(u01_f(r.v[0])));
            sincos2pi_f(u01_f(r.v[1]), &sn, &cs);
            N[0] = rad * cs; N[1] = rad * sn;
            rad = std::sqrt(-2.0f * log_f(u01_f(r.v[2])));
            sincos2pi_f(u01_f(r.v[3]), &sn, &cs);
            N[2] = rad * cs; N[3] = rad * sn;
        } else {
            double sn, cs;
            double rad = std::sqrt(-2.0 * log_d(u01_d(r.v[0])));
            sincos2pi_d(u01_d(r.v[1]), &sn, &cs);
            N[0] = rad * cs; N[1] = rad * sn;
            rad = std::sqrt(-2.0 * log_d(u01_d(r.v[2])));
            sincos2pi_d(u01_d(r.v[3]), &sn, &cs);
            N[2] = rad * cs; N[3] = rad * sn;
        }
        for (int i = 0; i < 4 && 4 * j + i < K; ++i) {
            const Real si = sig * N[i];
            e = e + si * si;
        }
    }
    return e;
}

// Tracking planes of every tet.  In the mixed mode (binary32 particles, reading)
// a particle's position is stored relative to the anchor of its tet: vertex 0
// rounded to the grid 2^-q with q = 22 - r, 2^r bounding the coordinates, so
// that anchors and their differences are exact in binary32 while offsets stay
// within about a cell of zero; the planes of a tet are written in its frame.
// In binary64 the anchors are 0 (global coordinates).
template <class Real> struct Planes {
    std::vector<Real> n;  // [4*nc][3]
    std::vector<Real> d;  // [4*nc]
    std::vector<int32_t> nb;  // [4*nc]: (tet << 2 | local face) or -1 - face for boundary
    std::vector<double> A;    // [3*nc] anchor of each tet
    std::vector<float> Af;    // [3*nc] the same, binary32 (exact)
    void build(const Geom& g) {
        n.resize(12 * (size_t)g.nc); d.resize(4 * (size_t)g.nc); nb.resize(4 * (size_t)g.nc);
        A.assign(3 * (size_t)g.nc, 0.0);
        Af.assign(3 * (size_t)g.nc, 0.0f);
        if (std::is_same<Real, float>::value) {
            double mx = 0.0;
            for (double v : g.xyz) mx = std::max(mx, std::fabs(v));
            int r = 0;
            while (std::ldexp(1.0, r) <= mx) ++r;
            const int q = 22 - r;
            for (int i = 0; i < g.nc; ++i)
                for (int c = 0; c < 3; ++c) {
                    const double v = g.xyz[3 * (size_t)g.tet[4 * i] + c];
                    A[3 * (size_t)i + c] = std::ldexp(std::nearbyint(std::ldexp(v, q)), -q);
                    Af[3 * (size_t)i + c] = (float)A[3 * (size_t)i + c];
                }
        }
        for (int i = 0; i < g.nc; ++i)
            for (int k = 0; k < 4; ++k) {
                int f = g.tet_face[4 * i + k];
                int sg = g.tet_sign[4 * i + k];
                for (int c = 0; c < 3; ++c) {
                    Real v = (Real)g.f_n[3 * (size_t)f + c];
                    n[12 * (size_t)i + 3 * k + c] = sg > 0 ? v : -v;
                }
                // the plane offset in the tet's frame: d - n.A in binary64
                const double* fn = &g.f_n[3 * (size_t)f];
                const double* Ai = &A[3 * (size_t)i];
                const double dl = g.f_d[f] - ((fn[0] * Ai[0] + fn[1] * Ai[1]) + fn[2] * Ai[2]);
                Real dv = (Real)dl;
                d[4 * (size_t)i + k] = sg > 0 ? dv : -dv;
                if (g.f_nbr[f] < 0) nb[4 * (size_t)i + k] = -1 - f;
                else if (sg > 0) nb[4 * (size_t)i + k] = (g.f_nbr[f] << 2) | g.f_nbr_k[f];
                else nb[4 * (size_t)i + k] = (g.f_owner[f] << 2) | g.f_owner_k[f];
            }
    }
};

struct TrackOut { int status; int cell; int ncross; int nwall; };
enum { ST_COLL = 1, ST_EXIT = 2, ST_LOST = 4 };

// Ballistic streaming x* = x + u t (Sec. 2.2) through the tets.  The particle
// follows the ray x0 + u (t - t0); in its tet the exit face is the one with
// u.n > 0 and the smallest crossing time (ties: lowest local face; the face it
// entered through, or last reflected from, is skipped).  Interior faces hand
// the ray to the neighbour unchanged (in the mixed mode moved into the
// neighbour's frame); walls restart it at the hit point.
template <class Real>
static TrackOut track(const Geom& g, const Planes<Real>& pl, const orc_params& P,
                      Part<Real>& pt, Real t_end, uint64_t step) {
    TrackOut o = {0, pt.cell, 0, 0};
    int tet = pt.cell, last = -1;
    Real x0[3] = {pt.x[0], pt.x[1], pt.x[2]};
    Real u[3] = {pt.u[0], pt.u[1], pt.u[2]};
    Real t0 = 0;
    for (;;) {
        // exit face: the smallest crossing time (d_k - n_k.x0)/(u.n_k) over the
        // faces with u.n_k > 0, compared as (d_k - n_k.x0)(u.n_j) <
        // (d_j - n_j.x0)(u.n_k) (both denominators positive); ties keep the
        // lower local face; the chosen time is one division
        int best = -1;
        Real nbest = 0, dbest = 1;
        for (int k = 0; k < 4; ++k) {
            if (k == last) continue;
            const Real* nk = &pl.n[12 * (size_t)tet + 3 * k];
            Real un = (u[0] * nk[0] + u[1] * nk[1]) + u[2] * nk[2];
            if (un > (Real)0) {
                Real xn = (x0[0] * nk[0] + x0[1] * nk[1]) + x0[2] * nk[2];
                Real num = pl.d[4 * (size_t)tet + k] - xn;
                if (best < 0 || num * dbest < nbest * un) { best = k; nbest = num; dbest = un; }
            }
        }
        Real sbest = best >= 0 ? nbest / dbest : (Real)0;
        Real rem = t_end - t0;
        if (best < 0 || sbest >= rem) {
            for (int c = 0; c < 3; ++c) pt.x[c] = x0[c] + u[c] * rem;
            break;
        }
        if (sbest < (Real)0) sbest = 0;
        o.ncross++;
        if (o.ncross > P.max_crossings) {
            o.status |= ST_LOST;
            for (int c = 0; c < 3; ++c) pt.x[c] = x0[c];
            break;
        }
        int code = pl.nb[4 * (size_t)tet + best];
        if (code >= 0) {
            const int nt = code >> 2;
            // mixed mode: the segment start moves into the frame of the next tet
            // (the anchor difference is exact in binary32)
            if (std::is_same<Real, float>::value)
                for (int c = 0; c < 3; ++c)
                    x0[c] = x0[c] + (Real)(pl.Af[3 * (size_t)tet + c] - pl.Af[3 * (size_t)nt + c]);
            tet = nt;
            last = code & 3;
            continue;
        }
        int f = -1 - code;
        const orc_bc& bc = P.bc[g.f_bc[f]];
        if (bc.type == ORC_BC_INFLOW || bc.type == ORC_BC_OUTFLOW) { o.status |= ST_EXIT; break; }
        Real xh[3];
        for (int c = 0; c < 3; ++c) xh[c] = x0[c] + u[c] * sbest;
        if (bc.type == ORC_BC_SPECULAR) {
            const Real* nk = &pl.n[12 * (size_t)tet + 3 * best];
            Real un = (u[0] * nk[0] + u[1] * nk[1]) + u[2] * nk[2];
            Real two = un + un;
            for (int c = 0; c < 3; ++c) u[c] = u[c] - two * nk[c];
        } else {
            // Diffuse re-emission with full accommodation (reading): flux-weighted
            // normal speed sqrt(-2 R T_w ln eta), Gaussian tangential components.
            Ctr4 r = draw(P.seed, pt.id, step, TAG_WALL, (uint64_t)o.nwall);
            if constexpr (std::is_same<Real, float>::value) {
                // mixed precision: binary32 arithmetic from the wall constants,
                // the face frame and U_w.t rounded to binary32
                const float c2 = (float)(-2.0 * P.R * bc.T_w);
                const float sw = (float)std::sqrt(P.R * bc.T_w);
                float vn = std::sqrt(c2 * log_f(u01_f(r.v[0])));
                float rad = std::sqrt(-2.0f * log_f(u01_f(r.v[1])));
                float sn, cs;
                sincos2pi_f(u01_f(r.v[2]), &sn, &cs);
                const double* n = &g.f_n[3 * (size_t)f];
                const double* t1 = &g.f_t1[3 * (size_t)f];
                const double* t2 = &g.f_t2[3 * (size_t)f];
                float v1 = (float)dot3(bc.U_w, t1) + sw * (rad * cs);
                float v2 = (float)dot3(bc.U_w, t2) + sw * (rad * sn);
                for (int c = 0; c < 3; ++c) u[c] = ((-vn) * (float)n[c] + v1 * (float)t1[c]) + v2 * (float)t2[c];
                if (P.K > 0) pt.e = internal_energy<float>(P.seed, pt.id, step, TAG_WINT, 2 * (uint64_t)o.nwall, P.K, sw);
            } else {
                double vn = std::sqrt(-2.0 * P.R * bc.T_w * log_d(u01_d(r.v[0])));
                double rad = std::sqrt(-2.0 * log_d(u01_d(r.v[1])));
                double sn, cs;
                sincos2pi_d(u01_d(r.v[2]), &sn, &cs);
                double sw = std::sqrt(P.R * bc.T_w);
                const double* n = &g.f_n[3 * (size_t)f];
                const double* t1 = &g.f_t1[3 * (size_t)f];
                const double* t2 = &g.f_t2[3 * (size_t)f];
                double v1 = dot3(bc.U_w, t1) + sw * (rad * cs);
                double v2 = dot3(bc.U_w, t2) + sw * (rad * sn);
                for (int c = 0; c < 3; ++c) u[c] = (Real)(((-vn) * n[c] + v1 * t1[c]) + v2 * t2[c]);
                if (P.K > 0)
                    pt.e = (Real)internal_energy<double>(P.seed, pt.id, step, TAG_WINT, 2 * (uint64_t)o.nwall, P.K, sw);
            }
            o.nwall++;
        }
        for (int c = 0; c < 3; ++c) x0[c] = xh[c];
        t0 = t0 + sbest;
        last = best;
    }
    o.cell = tet;
    for (int c = 0; c < 3; ++c) pt.u[c] = u[c];
    return o;
}

// Fixed-point image of phi = m (1, u, |u|^2/2) (Sec. 2.2, Eq. W^p): each
// component scaled by its power-of-two quantum 2^e and rounded to nearest even.
template <class Real>
static bool phi_fixed(const Part<Real>& pt, const int* e, int64_t q[5]) {
    double u0 = (double)pt.u[0], u1 = (double)pt.u[1], u2 = (double)pt.u[2];
    double m = pt.m;
    double phi[5] = {m, m * u0, m * u1, m * u2, 0.5 * (m * (((u0 * u0 + u1 * u1) + u2 * u2) + (double)pt.e))};
    bool ok = true;
    for (int k = 0; k < 5; ++k) {
        double v = std::ldexp(phi[k], -e[k]);
        if (!(std::fabs(v) < 0x1p62)) { ok = false; v = 0.0; }
        q[k] = std::llrint(v);
    }
    return ok;
}

// ------------------------------------------------------------ simulation
struct SimBase {
    Geom g;
    orc_params P;
    std::vector<double> W;  // [5][nc]
    int64_t step = 0;
    double t = 0.0;
    int e[5] = {0, 0, 0, 0, 0};
    // diagnostics of the last step
    double dt = 0.0;
    std::vector<double> tau, rhoh, msam, F;
    std::vector<int64_t> nsam, pflux, smass, scount;
    int64_t counters[7] = {0, 0, 0, 0, 0, 0, 0};
    virtual ~SimBase() {}
    virtual int64_t n_particles() const = 0;
    virtual int do_step(std::string& err) = 0;
    virtual int prepare(std::string& err) = 0;
    virtual int64_t sample_one_cell(int cell, int64_t cap, uint64_t* id, double* x, double* u, double* m,
                                    double* e) const = 0;
    virtual bool gp_coef(int cell, double* out) const = 0;
    virtual void get_particles(uint64_t*, int32_t*, double*, double*, double*, double*) const = 0;
    virtual bool set_particles(int64_t, const uint64_t*, const int32_t*, const double*, const double*,
                               const double*, const double*, std::string&) = 0;
    virtual int track_one(uint64_t, int32_t, double*, double*, double*, double, double, int64_t, int32_t*, int32_t*) const = 0;
    // a3 (order 2): limited least-squares gradients of W and rho^h; a4: the
    // time-integrated wave flux F of every face from W and rho^h, over dt or,
    // when dtf is given, over dtf[f].  gks: no particles (both halves of the
    // free transport carry q4, q5).
    void face_fluxes(bool gks, const std::vector<double>* dtf) {
        const int nc = g.nc, nf = g.nf;
        const orc_params& p = P;
        std::vector<double> gW, gH;
        if (p.order == 2) limited_gradients(g, p, W, rhoh, true, gW, gH);
        F.assign(5 * (size_t)nf, 0.0);
        for (int f = 0; f < nf; ++f) {
            const double* n = &g.f_n[3 * (size_t)f];
            const double dtv = dtf ? (*dtf)[f] : dt;
            int o = g.f_owner[f], nb = g.f_nbr[f];
            double WL[5], Fv[5];
            for (int k = 0; k < 5; ++k) WL[k] = W[(size_t)k * nc + o];
            if (nb >= 0 && p.order == 2) {
                double WR[5], dxL[3], dxR[3];
                for (int k = 0; k < 5; ++k) WR[k] = W[(size_t)k * nc + nb];
                const double* xf = &g.f_c[3 * (size_t)f];
                for (int d = 0; d < 3; ++d) {
                    dxL[d] = xf[d] - g.cen[3 * (size_t)o + d];
                    dxR[d] = xf[d] - g.cen[3 * (size_t)nb + d];
                }
                Frame R = frame_of(n);
                face_flux_o2(R, WL, rhoh[o], &gW[15 * (size_t)o], &gH[3 * (size_t)o], dxL, WR, rhoh[nb],
                             &gW[15 * (size_t)nb], &gH[3 * (size_t)nb], dxR, dtv, gks, p, Fv);
            } else if (nb >= 0) {
                double WR[5];
                for (int k = 0; k < 5; ++k) WR[k] = W[(size_t)k * nc + nb];
                FaceState L = face_state(WL, rhoh[o], n, p.R, p.K), Rs = face_state(WR, rhoh[nb], n, p.R, p.K);
                interior_flux(L, Rs, false, gks, n, dtv, p, Fv);
            } else {
                boundary_flux(WL, rhoh[o], tau[o], p.bc[g.f_bc[f]], n, dtv, gks, p, Fv);
            }
            for (int k = 0; k < 5; ++k) F[(size_t)k * nf + f] = Fv[k];
        }
    }

    // One step of the gas-kinetic scheme (GKS) that the method reduces to
    // without particles (Sec. 3.2), for the start-up fields of the steady cases
    // (Sec. 4.3, 4.4): W^h = W, nothing sampled, the whole free transport in the wave
    // flux.  local: local time stepping (reading) with dt_i = CFL |Omega_i| /
    // sum_d Lambda_i^d per cell, each face integrated over dt_f = the smaller
    // dt of its cells (the interior cell's at a boundary), and cell i advanced
    // by dt_i times the mean flux rate F_f / dt_f (which F then holds); t is
    // then left unchanged.
    int gks_step(bool local, std::string& err) {
        if (n_particles() != 0) { err = "a GKS step needs a state without particles"; return -10; }
        const int nc = g.nc, nf = g.nf;
        const orc_params& p = P;
        tau.assign(nc, 0.0); rhoh.assign(nc, 0.0);
        std::vector<double> dtc(nc, 0.0);
        double rmin = HUGE_VAL;
        for (int i = 0; i < nc; ++i) {
            double Wi[5];
            for (int k = 0; k < 5; ++k) Wi[k] = W[(size_t)k * nc + i];
            Prim s = prim_of(Wi, p.R, p.K);
            if (!(s.rho > 0.0) || !(s.p > 0.0) || !std::isfinite(s.p)) {
                err = "non-positive density or pressure in cell " + std::to_string(i);
                return -9;
            }
            tau[i] = tau_cell(s, p);
            rhoh[i] = s.rho;
            double c = 3.0 * std::sqrt(p.R * s.T);
            double lam = ((std::fabs(s.U[0]) + c) * g.dS[3 * i] + (std::fabs(s.U[1]) + c) * g.dS[3 * i + 1])
                       + (std::fabs(s.U[2]) + c) * g.dS[3 * i + 2];
            double r = g.vol[i] / lam;
            dtc[i] = p.CFL * r;
            if (r < rmin) rmin = r;
        }
        dt = p.CFL * rmin;
        std::vector<double> dtf;
        if (local) {
            dtf.assign(nf, 0.0);
            for (int f = 0; f < nf; ++f) {
                const int o = g.f_owner[f], nb = g.f_nbr[f];
                dtf[f] = nb >= 0 ? std::fmin(dtc[o], dtc[nb]) : dtc[o];
            }
        }
        face_fluxes(true, local ? &dtf : nullptr);
        if (local)  // F becomes the mean flux rate F_f / dt_f
            for (int q = 0; q < 5; ++q)
                for (int f = 0; f < nf; ++f) F[(size_t)q * nf + f] = F[(size_t)q * nf + f] / dtf[f];
        for (int i = 0; i < nc; ++i) {
            for (int q = 0; q < 5; ++q) {
                double s = 0.0;
                for (int k = 0; k < 4; ++k) {
                    int f = g.tet_face[4 * i + k];
                    double v = F[(size_t)q * nf + f] * g.f_area[f];
                    s = s + (g.tet_sign[4 * i + k] > 0 ? v : -v);
                }
                double& Wq = W[(size_t)q * nc + i];
                Wq = local ? Wq - (dtc[i] * s) / g.vol[i] : Wq - s / g.vol[i];
            }
        }
        if (!local) t += dt;
        return 0;
    }
};

template <class Real> struct Sim : SimBase {
    Planes<Real> pl;
    std::vector<Part<Real>> parts;

    int64_t n_particles() const override { return (int64_t)parts.size(); }

    // per-cell quantities of the current state (a1, a2, a5 counts)
    std::vector<Prim> pr;
    std::vector<double> rho_p;
    std::vector<int64_t> nleft;
    // first-order g_p sampling: per cell the polynomial phi(X) of the
    // acceptance weight 1 + phi and its bound (GP_NC values, see gp_coefficients)
    std::vector<double> gpc;

    // a1 + a2 + sampling counts for the current state; no state change.
    int prepare(std::string& err) override {
        const int nc = g.nc;
        const orc_params& p = P;
        // ---- a1: primitives and relaxation time; W^h density = W - W^p (Sec. 2.2)
        pr.assign(nc, Prim());
        tau.assign(nc, 0.0); rhoh.assign(nc, 0.0);
        std::vector<int64_t> mass_q(nc, 0);
        nleft.assign(nc, 0);
        for (const auto& pt : parts) {
            int64_t q[5];
            phi_fixed(pt, e, q);
            mass_q[pt.cell] += q[0];
            nleft[pt.cell] += 1;
        }
        rho_p.assign(nc, 0.0);
        for (int i = 0; i < nc; ++i) {
            double Wi[5];
            for (int k = 0; k < 5; ++k) Wi[k] = W[(size_t)k * nc + i];
            pr[i] = prim_of(Wi, p.R, p.K);
            if (!(pr[i].rho > 0.0) || !(pr[i].p > 0.0) || !std::isfinite(pr[i].p)) {
                err = "non-positive density or pressure in cell " + std::to_string(i);
                return -9;
            }
            tau[i] = tau_cell(pr[i], p);
            rho_p[i] = std::ldexp((double)mass_q[i], e[0]) / g.vol[i];
            rhoh[i] = pr[i].rho - rho_p[i];
        }
        // ---- a2: time step (Sec. 2.4 (a)), c = 3 sqrt(RT)
        double rmin = HUGE_VAL;
        for (int i = 0; i < nc; ++i) {
            double c = 3.0 * std::sqrt(p.R * pr[i].T);
            double lam = ((std::fabs(pr[i].U[0]) + c) * g.dS[3 * i] + (std::fabs(pr[i].U[1]) + c) * g.dS[3 * i + 1])
                       + (std::fabs(pr[i].U[2]) + c) * g.dS[3 * i + 2];
            double r = g.vol[i] / lam;
            if (r < rmin) rmin = r;
        }
        dt = p.CFL * rmin;
        // ---- a5 counts (Sec. 2.4 (b)): rho^hp = e^{-dt/tau} rho^h, m_ref, N_sam, m_sam
        nsam.assign(nc, 0); msam.assign(nc, 0.0);
        for (int i = 0; i < nc; ++i) {
            double ex = exp_d(-(dt / tau[i]));
            double rh = rhoh[i] > 0.0 ? rhoh[i] : 0.0;  // reading: clamp noise-negative rho^h
            double rhp = ex * rh;
            double Mhp = rhp * g.vol[i];
            if (!(Mhp > (pr[i].rho * g.vol[i]) * 0x1p-30)) continue;  // reading: below noise floor
            double mref = ((rho_p[i] + rhp) * g.vol[i]) / (double)p.N_ref;
            int64_t ns = 2 * (int64_t)std::ceil(Mhp / (2.0 * mref));
            int64_t need = (int64_t)p.N_min - nleft[i];
            if (need > ns) ns = need + (need & 1);
            if (ns > 65534) { err = "more than 65534 particles sampled in one cell"; return -6; }
            nsam[i] = ns;
            msam[i] = Mhp / (double)ns;
        }
        if (p.sampling == 2) {
            std::vector<double> gW, gH;
            limited_gradients(g, p, W, rhoh, true, gW, gH);
            gpc.assign(GP_NC * (size_t)nc, 0.0);
            for (int i = 0; i < nc; ++i) gp_coefficients(pr[i], &gW[15 * (size_t)i], tau[i], dt, P.R, &gpc[GP_NC * (size_t)i]);
        }
        return 0;
    }

    // First-order g_p draws in the particle precision, widened.
    void gp_normals(const double* c, uint64_t id, double Xout[3]) const {
        gp_draw<Real>(P.seed, (uint64_t)step, c, id, Xout);
    }

    // a5 positions (reading): three uniforms N_k 2^-48 with N_k odd and below
    // 2^48 (the top 47 bits of a Philox word, doubled, plus one), folded from
    // the cube to the prism to the tet (Rocchini and Cignoni, J. Graphics Tools
    // 5(4), 2000) on the integers N_k, so that both modes place the particle
    // with the same exact barycentric weights.
    static void fold_weights(const Ctr4& r, int64_t N[3]) {
        const int64_t one = (int64_t)1 << 48;
        int64_t a = (int64_t)(((r.v[0] >> 17) << 1) | 1), b = (int64_t)(((r.v[1] >> 17) << 1) | 1);
        int64_t c = (int64_t)(((r.v[2] >> 17) << 1) | 1);
        if (a + b > one) { a = one - a; b = one - b; }
        if (b + c > one) { int64_t t = c; c = one - a - b; b = one - t; }
        else if (a + b + c > one) { int64_t t = c; c = a + b + c - one; a = one - b - t; }
        N[0] = a; N[1] = b; N[2] = c;
    }

    // a binary64 value as the binary32 pair (value rounded, remainder rounded)
    static void split32(double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }

    // Knuth's exact sum: s + e equals a + b
    static void exact_sum(float a, float b, float& s, float& e) {
        s = a + b;
        float v = s - a;
        e = (a - (s - v)) + (b - v);
    }

    // Mixed mode: one coordinate of the position offset from the tet's anchor,
    // (p0 - A) + ((w1 e1 + w2 e2) + w3 e3) carried on binary32 pairs and
    // rounded to binary32 at the end.  A product w e keeps its high parts'
    // rounding error exactly (fused multiply-add) plus the two cross terms;
    // each sum keeps its exact error in the low part.
    static float offset_on_pairs(double p0A, const double e[3], const int64_t N[3]) {
        float ph[3], pe[3];
        for (int k = 0; k < 3; ++k) {
            const float wh = (float)(N[k] >> 24) * 0x1p-24f, wl = (float)(N[k] & 0xffffff) * 0x1p-48f;
            float eh, el;
            split32(e[k], eh, el);
            ph[k] = wh * eh;
            pe[k] = std::fmaf(wh, eh, -ph[k]) + (wh * el + wl * eh);
        }
        float s, r;
        exact_sum(ph[0], ph[1], s, r);
        float low = r + (pe[0] + pe[1]);
        float s2, r2;
        exact_sum(s, ph[2], s2, r2);
        low = r2 + (low + pe[2]);
        float ah, al;
        split32(p0A, ah, al);
        float s3, r3;
        exact_sum(ah, s2, s3, r3);
        low = r3 + (low + al);
        return s3 + low;
    }

    // The three normals X of the pair whose first member has id `ida`, by
    // Box-Muller in the particle precision (binary32 in the mixed mode), widened.
    static void normals_of_pair(uint64_t seed, uint64_t step, uint64_t ida, double X[3]) {
        Ctr4 r = draw(seed, ida, step, TAG_SVEL, 0);
        if constexpr (std::is_same<Real, float>::value) {
            float sn, cs;
            float rad = std::sqrt(-2.0f * log_f(u01_f(r.v[0])));
            sincos2pi_f(u01_f(r.v[1]), &sn, &cs);
            X[0] = (double)(rad * cs); X[1] = (double)(rad * sn);
            rad = std::sqrt(-2.0f * log_f(u01_f(r.v[2])));
            sincos2pi_f(u01_f(r.v[3]), &sn, &cs);
            X[2] = (double)(rad * cs);
        } else {
            double sn, cs;
            double rad = std::sqrt(-2.0 * log_d(u01_d(r.v[0])));
            sincos2pi_d(u01_d(r.v[1]), &sn, &cs);
            X[0] = rad * cs; X[1] = rad * sn;
            rad = std::sqrt(-2.0 * log_d(u01_d(r.v[2])));
            sincos2pi_d(u01_d(r.v[3]), &sn, &cs);
            X[2] = rad * cs;
        }
    }

    // a5: the N_sam particles of cell i, in pairs u = U +/- sqrt(RT) X with
    // X ~ N(0, I) (Box-Muller), x uniform in the tet (needs prepare()).  The
    // binary64 mode draws in binary64.  The mixed mode (reading) draws the
    // velocities in binary32 from U and sqrt(RT) rounded to binary32, and the
    // position offset from the tet's anchor on binary32 pairs, rounded once.
    void sample_cell(int i, std::vector<Part<Real>>& out) const {
        const orc_params& p = P;
        const int64_t ns = nsam[i];
        const double ms = msam[i];
        double sig = std::sqrt(p.R * pr[i].T);
        const double *p0 = &g.xyz[3 * (size_t)g.tet[4 * i]], *p1 = &g.xyz[3 * (size_t)g.tet[4 * i + 1]];
        const double *p2 = &g.xyz[3 * (size_t)g.tet[4 * i + 2]], *p3 = &g.xyz[3 * (size_t)g.tet[4 * i + 3]];
        constexpr bool mixed = std::is_same<Real, float>::value;
        // Energy-matched sampling (option): one factor s for all pairs of the
        // cell so that the sampled thermal energy sum_j m (s sqrt(RT))^2 |X_j|^2
        // equals N_sam m (3/2) R T exactly, i.e. s^2 sum_j |X_j|^2 = 3 N_sam / 2
        // (the X of the particle precision, summed in binary64).
        if (p.sampling == 1 && ns >= 2) {
            double S = 0.0;
            for (int64_t j = 0; j < ns / 2; ++j) {
                double X[3];
                normals_of_pair(p.seed, (uint64_t)step, make_id((uint64_t)step, (uint64_t)i, (uint64_t)(2 * j)), X);
                S = S + ((X[0] * X[0] + X[1] * X[1]) + X[2] * X[2]);
            }
            if (S > 0.0) sig = sig * std::sqrt((double)(3 * (ns / 2)) / S);
        }
        const float Uf[3] = {(float)pr[i].U[0], (float)pr[i].U[1], (float)pr[i].U[2]};
        const float sigf = (float)sig;
        for (int64_t j = 0; j < ns / 2; ++j) {
            uint64_t ida = make_id((uint64_t)step, (uint64_t)i, (uint64_t)(2 * j));
            double X[3];
            normals_of_pair(p.seed, (uint64_t)step, ida, X);
            for (int side = 0; side < 2; ++side) {
                Part<Real> pt;
                pt.id = ida + (uint64_t)side;
                pt.cell = i;
                pt.m = ms;
                double Xs[3] = {X[0], X[1], X[2]};
                if (p.sampling == 2) gp_normals(&gpc[GP_NC * (size_t)i], pt.id, Xs);  // every particle on its own
                const bool plus = p.sampling == 2 || side == 0;
                for (int c = 0; c < 3; ++c) {
                    if constexpr (mixed) {
                        const float xs = (float)Xs[c];
                        pt.u[c] = plus ? Uf[c] + sigf * xs : Uf[c] - sigf * xs;
                    } else {
                        pt.u[c] = plus ? pr[i].U[c] + sig * Xs[c] : pr[i].U[c] - sig * Xs[c];
                    }
                }
                if (p.K > 0) {
                    if constexpr (mixed) pt.e = internal_energy<float>(p.seed, pt.id, (uint64_t)step, TAG_SINT, 0, p.K, sigf);
                    else pt.e = internal_energy<double>(p.seed, pt.id, (uint64_t)step, TAG_SINT, 0, p.K, sig);
                }
                int64_t N[3];
                fold_weights(draw(p.seed, pt.id, (uint64_t)step, TAG_SPOS, 0), N);
                for (int c = 0; c < 3; ++c) {
                    const double e[3] = {p1[c] - p0[c], p2[c] - p0[c], p3[c] - p0[c]};
                    if constexpr (mixed) {
                        pt.x[c] = offset_on_pairs(p0[c] - pl.A[3 * (size_t)i + c], e, N);
                    } else {
                        const double a = (double)N[0] * 0x1p-48, b = (double)N[1] * 0x1p-48, cc = (double)N[2] * 0x1p-48;
                        pt.x[c] = p0[c] + ((a * e[0] + b * e[1]) + cc * e[2]);
                    }
                }
                out.push_back(pt);
            }
        }
    }

    int do_step(std::string& err) override {
        const int nc = g.nc, nf = g.nf;
        const orc_params& p = P;
        int prc = prepare(err);
        if (prc) return prc;
        // ---- a5: sample the collisionless part of the hydrodynamic wave
        const size_t n_old = parts.size();
        int64_t n_sampled = 0;
        for (int i = 0; i < nc; ++i) {
            if (!nsam[i]) continue;
            sample_cell(i, parts);
            n_sampled += nsam[i];
        }
        // ---- a6..a9: free-transport time (Eq. t_f), streaming, counting flux
        // F^{fr,p}_i = sum_{end in i} phi - sum_{start in i} phi (Sec. 2.3),
        // removal of collisional (t_f < dt) and exited particles (Sec. 2.2).
        pflux.assign(5 * (size_t)nc, 0);
        smass.assign(nc, 0); scount.assign(nc, 0);
        const Real dtR = (Real)dt;
        std::vector<Part<Real>> kept;
        kept.reserve(parts.size());
        int64_t ncoll = 0, nexit = 0, nlost = 0, ncross = 0, nwall = 0;
        bool overflow = false;
        for (size_t k = 0; k < parts.size(); ++k) {
            Part<Real> pt = parts[k];
            int64_t q0[5], q1[5];
            overflow |= !phi_fixed(pt, e, q0);
            const int c0 = pt.cell;
            Real t_end = dtR;
            bool coll = false;
            if (k < n_old) {
                const uint64_t r = draw_tf(p.seed, pt.id, (uint64_t)step);
                Real tf;
                if (sizeof(Real) == 8) tf = (Real)(-((double)tau[c0] * log_d(u01_d(r))));
                else tf = (Real)(-((float)tau[c0] * log_f(u01_f(r))));
                if (tf < dtR) { coll = true; t_end = tf; }
            }
            TrackOut o = track<Real>(g, pl, p, pt, t_end, (uint64_t)step);
            ncross += o.ncross; nwall += o.nwall;
            for (int c = 0; c < 5; ++c) pflux[(size_t)c * nc + c0] -= q0[c];
            if (o.status & ST_EXIT) { nexit++; continue; }
            if (o.status & ST_LOST) nlost++;
            pt.cell = o.cell;
            overflow |= !phi_fixed(pt, e, q1);
            for (int c = 0; c < 5; ++c) pflux[(size_t)c * nc + o.cell] += q1[c];
            if (coll && !(o.status & ST_LOST)) { ncoll++; continue; }
            smass[o.cell] += q1[0];
            scount[o.cell] += 1;
            kept.push_back(pt);
        }
        counters[0] = (int64_t)parts.size(); counters[1] = ncoll; counters[2] = nexit;
        counters[3] = nlost; counters[4] = ncross; counters[5] = nwall; counters[6] = n_sampled;
        parts.swap(kept);
        // ---- a3 (order 2) + a4: wave flux per face from W^n and rho^{h,n}
        face_fluxes(false, nullptr);
        // ---- a10: W^{n+1} = W^n - 1/|Omega| sum_j (F^eq + F^{fr,wave}) |S| + F^{fr,p}/|Omega|
        for (int i = 0; i < nc; ++i) {
            for (int q = 0; q < 5; ++q) {
                double s = 0.0;
                for (int k = 0; k < 4; ++k) {
                    int f = g.tet_face[4 * i + k];
                    double v = F[(size_t)q * nf + f] * g.f_area[f];
                    s = s + (g.tet_sign[4 * i + k] > 0 ? v : -v);
                }
                double fp = std::ldexp((double)pflux[(size_t)q * nc + i], e[q]);
                double& Wq = W[(size_t)q * nc + i];
                Wq = (Wq - s / g.vol[i]) + fp / g.vol[i];
            }
        }
        step += 1;
        t += dt;
        if (overflow) { err = "fixed-point overflow"; return -8; }
        if (nlost) { err = std::to_string(nlost) + " particles exceeded max_crossings"; return -7; }
        return 0;
    }

    bool gp_coef(int cell, double* out) const override {
        if (gpc.size() != GP_NC * (size_t)g.nc) return false;
        for (int k = 0; k < GP_NC; ++k) out[k] = gpc[GP_NC * (size_t)cell + k];
        return true;
    }

    int64_t sample_one_cell(int cell, int64_t cap, uint64_t* id, double* x, double* u, double* m,
                            double* e) const override {
        std::vector<Part<Real>> v;
        sample_cell(cell, v);
        const int64_t n = (int64_t)v.size();
        for (int64_t k = 0; k < n && k < cap; ++k) {
            id[k] = v[k].id;
            m[k] = v[k].m;
            if (e) e[k] = (double)v[k].e;
            for (int c = 0; c < 3; ++c) {
                x[3 * k + c] = pl.A[3 * (size_t)cell + c] + (double)v[k].x[c];
                u[3 * k + c] = (double)v[k].u[c];
            }
        }
        return n;
    }

    void get_particles(uint64_t* id, int32_t* cell, double* x, double* u, double* m, double* e) const override {
        size_t n = parts.size();
        for (size_t k = 0; k < n; ++k) {
            const auto& pt = parts[k];
            if (id) id[k] = pt.id;
            if (cell) cell[k] = pt.cell;
            // positions: anchor + offset (exact in binary64)
            for (int c = 0; c < 3; ++c) {
                if (x) x[c * n + k] = pl.A[3 * (size_t)pt.cell + c] + (double)pt.x[c];
                if (u) u[c * n + k] = (double)pt.u[c];
            }
            if (m) m[k] = pt.m;
            if (e) e[k] = (double)pt.e;
        }
    }

    bool set_particles(int64_t n, const uint64_t* id, const int32_t* cell, const double* x,
                       const double* u, const double* m, const double* e, std::string& err) override {
        parts.resize((size_t)n);
        for (int64_t k = 0; k < n; ++k) {
            Part<Real>& pt = parts[(size_t)k];
            pt.id = id[k]; pt.cell = cell[k]; pt.m = m[k];
            if (pt.cell < 0 || pt.cell >= g.nc) { err = "particle cell out of range"; return false; }
            for (int c = 0; c < 3; ++c) {
                const double xl = x[c * n + k] - pl.A[3 * (size_t)pt.cell + c];
                pt.x[c] = (Real)xl;
                pt.u[c] = (Real)u[c * n + k];
                if ((double)pt.x[c] != xl || pl.A[3 * (size_t)pt.cell + c] + xl != x[c * n + k] ||
                    (double)pt.u[c] != u[c * n + k]) {
                    err = "particle state not representable in the particle precision"; return false;
                }
            }
            pt.e = (Real)0;
            if (e && P.K > 0) {
                pt.e = (Real)e[k];
                if ((double)pt.e != e[k] || !(e[k] >= 0.0)) {
                    err = "internal energy negative or not representable in the particle precision"; return false;
                }
            }
        }
        return true;
    }

    int track_one(uint64_t id, int32_t cell, double* io_x, double* io_u, double* io_e, double tau_c, double dtv,
                  int64_t stp, int32_t* cell_out, int32_t* nc_out) const override {
        Part<Real> pt;
        pt.id = id; pt.cell = cell; pt.m = 1.0;
        for (int c = 0; c < 3; ++c) {
            pt.x[c] = (Real)(io_x[c] - pl.A[3 * (size_t)cell + c]);
            pt.u[c] = (Real)io_u[c];
        }
        if (io_e) pt.e = (Real)*io_e;
        const Real dtR = (Real)dtv;
        Real t_end = dtR;
        int st = 0;
        if (id_step(id) != (uint64_t)stp) {
            const uint64_t r = draw_tf(P.seed, id, (uint64_t)stp);
            Real tf;
            if (sizeof(Real) == 8) tf = (Real)(-(tau_c * log_d(u01_d(r))));
            else tf = (Real)(-((float)tau_c * log_f(u01_f(r))));
            if (tf < dtR) { st |= ST_COLL; t_end = tf; }
        }
        TrackOut o = track<Real>(g, pl, P, pt, t_end, (uint64_t)stp);
        for (int c = 0; c < 3; ++c) {
            io_x[c] = pl.A[3 * (size_t)o.cell + c] + (double)pt.x[c];
            io_u[c] = (double)pt.u[c];
        }
        if (io_e) *io_e = (double)pt.e;
        *cell_out = o.cell;
        *nc_out = o.ncross;
        return st | o.status;
    }
};

// Fixed-point quanta 2^e_q (reading): e_q = ceil(log2 B_q) - 50 with
// B_mass = max_i rho_i |Omega_i|, B_mom = B_mass c, B_E = B_mass c^2 / 2 and
// c = max over cells and boundary states of |U| + 5 sqrt(RT).
static int ceil_log2(double b) {
    int ex;
    double mant = std::frexp(b, &ex);
    return mant == 0.5 ? ex - 1 : ex;
}
static void scale_exponents(const Geom& g, const orc_params& P, const std::vector<double>& W, int e[5]) {
    double bm = 0.0, cmax = 0.0;
    int nc = g.nc;
    for (int i = 0; i < nc; ++i) {
        double Wi[5];
        for (int k = 0; k < 5; ++k) Wi[k] = W[(size_t)k * nc + i];
        Prim s = prim_of(Wi, P.R, P.K);
        double mass = s.rho * g.vol[i];
        if (mass > bm) bm = mass;
        double c = std::sqrt(dot3(s.U, s.U)) + 5.0 * std::sqrt(P.R * s.T);
        if (c > cmax) cmax = c;
    }
    for (int b = 0; b < P.n_bc; ++b) {
        const orc_bc& bc = P.bc[b];
        if (bc.type == ORC_BC_DIFFUSE_WALL) {
            double c = std::sqrt(dot3(bc.U_w, bc.U_w)) + 5.0 * std::sqrt(P.R * bc.T_w);
            if (c > cmax) cmax = c;
        } else if (bc.type == ORC_BC_INFLOW) {
            Prim s = prim_of(bc.W_in, P.R, P.K);
            double c = std::sqrt(dot3(s.U, s.U)) + 5.0 * std::sqrt(P.R * s.T);
            if (c > cmax) cmax = c;
        }
    }
    e[0] = ceil_log2(bm) - 50;
    e[1] = e[2] = e[3] = ceil_log2(bm * cmax) - 50;
    e[4] = ceil_log2(bm * cmax * cmax * 0.5) - 50;
}

}  // namespace orc

using namespace orc;

// --------------------------------------------- frozen-particle wave map
// The wave part of the step with the particle part frozen (first order): from
// W^0, for n = 0..K-1,
//   W^{n+1}_i = W^n_i - sum_f (+/-) F_f(W^n) |S_f| / |Omega_i| + pf^n_i / |Omega_i|
// with the recorded time steps dt^n, particle densities rho^p_n (so that
// rho^h = rho - rho^p) and particle fluxes pf^n (Sec. 2.3 update with
// F^{fr,p} a constant).  The face fluxes are those of the step (Sec. 2.1, 2.3,
// 2.4 (d), (e)), written once more here generic in the scalar type so that
// the same code gives the value (double) and forward-mode derivatives (Dual).
// Parameters theta = (rho_inf, U_inf, T_w): every far-field condition whose
// state equals the first far-field state becomes the Maxwellian of density
// rho_inf and speed U_inf along that state's velocity direction (x if it is
// at rest) at its own temperature; every diffuse wall whose tag is listed
// gets the temperature T_w.  J = sum_n sum_{faces with a listed tag}
// F_f[c] |S_f|, c = 1 (x momentum delivered to the walls: drag) or 4 (energy:
// wall heat flux), wave part only.
namespace frozen {

template <class S> struct PrimS { S rho, U[3], p, T, lam; };

template <class S> PrimS<S> prim_s(const S* W, double R) {
    PrimS<S> s;
    s.rho = W[0];
    for (int d = 0; d < 3; ++d) s.U[d] = W[1 + d] / s.rho;
    S U2 = (s.U[0] * s.U[0] + s.U[1] * s.U[1]) + s.U[2] * s.U[2];
    s.p = (W[4] - 0.5 * (s.rho * U2)) / 1.5;
    s.T = s.p / (s.rho * R);
    s.lam = s.rho / (2.0 * s.p);
    return s;
}

template <class S> S tau_cell_s(const PrimS<S>& s, const orc_params& P) {
    return (P.mu_ref / s.p) * exp_d(P.omega * log_d(s.T / P.T_ref));
}

// q1, q4, a4 = q4 - dt e^{-dt/tau}: series below x = dt/tau = 1, closed forms above
template <class S> void qcoef_s(double dt, const S& tau, S& q1, S& q4, S& a4) {
    S x = dt / tau;
    if (x < 1.0) {
        S s1 = 0.0, s4 = 0.0, sa = 0.0, term = 1.0;
        for (int k = 1; k <= 30; ++k) {
            term = term * x / (double)k;
            double sg = (k % 2 == 0) ? 1.0 : -1.0;
            if (k >= 2) s1 = s1 + sg * term;
            s4 = s4 + (-sg) * term;
            if (k >= 2) sa = sa + (-sg * (double)(1 - k)) * term;
        }
        q1 = tau * s1; q4 = tau * s4; a4 = tau * sa;
    } else {
        S e = exp(-x);
        S ph = -expm1(-x);
        q1 = dt - tau * ph;
        q4 = tau * ph;
        a4 = q4 - dt * e;
    }
}

template <class S> void un_moments_s(const S& Un, const S& lam, int half, S M[5]) {
    if (half == 0) {
        M[0] = 1.0; M[1] = Un;
    } else {
        S a = sqrt(lam) * Un;
        S edge = 0.5 * exp(-lam * Un * Un) / sqrt(PI * lam);
        if (half > 0) { M[0] = 0.5 * erfc(-a); M[1] = Un * M[0] + edge; }
        else          { M[0] = 0.5 * erfc(a);  M[1] = Un * M[0] - edge; }
    }
    for (int k = 0; k < 3; ++k) M[k + 2] = Un * M[k + 1] + (double)(k + 1) / (2.0 * lam) * M[k];
}

template <class S> void half_moments_s(const S& Un, const S* Ut, const double* n, const S& lam, int half,
                                      S H[5], S G[5]) {
    S M[5];
    un_moments_s(Un, lam, half, M);
    S Ut2 = (Ut[0] * Ut[0] + Ut[1] * Ut[1]) + Ut[2] * Ut[2];
    S tv = Ut2 + 1.0 / lam;
    H[0] = M[0];
    G[0] = M[1];
    for (int d = 0; d < 3; ++d) {
        H[1 + d] = M[1] * n[d] + M[0] * Ut[d];
        G[1 + d] = M[2] * n[d] + M[1] * Ut[d];
    }
    H[4] = 0.5 * (M[2] + M[0] * tv);
    G[4] = 0.5 * (M[3] + M[1] * tv);
}

template <class S> struct FaceS { S rho, rhoh, Un, Ut[3], lam, p, T; };

template <class S> FaceS<S> face_state_s(const S* W, const S& rhoh, const double* n, double R) {
    PrimS<S> s = prim_s(W, R);
    FaceS<S> f;
    f.rho = s.rho; f.rhoh = rhoh; f.lam = s.lam; f.p = s.p; f.T = s.T;
    f.Un = (s.U[0] * n[0] + s.U[1] * n[1]) + s.U[2] * n[2];
    for (int d = 0; d < 3; ++d) f.Ut[d] = s.U[d] - f.Un * n[d];
    return f;
}

template <class S> void interior_flux_s(const FaceS<S>& L, const FaceS<S>& Rs, bool ghost_hydro, const double* n,
                                       double dt, const orc_params& P, S F[5]) {
    S HL[5], GL[5], HR[5], GR[5];
    half_moments_s(L.Un, L.Ut, n, L.lam, +1, HL, GL);
    half_moments_s(Rs.Un, Rs.Ut, n, Rs.lam, -1, HR, GR);
    S W0[5];
    for (int q = 0; q < 5; ++q) W0[q] = L.rho * HL[q] + Rs.rho * HR[q];
    PrimS<S> s0 = prim_s(W0, P.R);
    S tau = P.mu_ref * pow(s0.T / P.T_ref, P.omega) / s0.p;
    if (P.C2 > 0.0) tau = tau + P.C2 * fabs(L.p - Rs.p) / fabs(L.p + Rs.p) * dt;
    S q1, q4, a4;
    qcoef_s(dt, tau, q1, q4, a4);
    S Un0 = (s0.U[0] * n[0] + s0.U[1] * n[1]) + s0.U[2] * n[2], Ut0[3];
    for (int d = 0; d < 3; ++d) Ut0[d] = s0.U[d] - Un0 * n[d];
    S H0[5], G0[5];
    half_moments_s(Un0, Ut0, n, s0.lam, 0, H0, G0);
    S cR = ghost_hydro ? q4 : a4;
    for (int k = 0; k < 5; ++k) F[k] = q1 * (s0.rho * G0[k]) + a4 * (L.rhoh * GL[k]) + cR * (Rs.rhoh * GR[k]);
}

template <class S> struct BcS { int type; S T_w; double U_w[3]; S W_in[5]; };

template <class S> void boundary_flux_s(const S* WL, const S& rhohL, const S& tauL, const BcS<S>& bc, const double* n,
                                       double dt, const orc_params& P, S F[5]) {
    FaceS<S> L = face_state_s(WL, rhohL, n, P.R);
    if (bc.type == ORC_BC_DIFFUSE_WALL) {
        S q1, q4, a4;
        qcoef_s(dt, tauL, q1, q4, a4);
        S HL[5], GL[5];
        half_moments_s(L.Un, L.Ut, n, L.lam, +1, HL, GL);
        S Gin[5];
        for (int k = 0; k < 5; ++k) Gin[k] = q1 * (L.rho * GL[k]) + a4 * (L.rhoh * GL[k]);
        S lamw = 1.0 / (2.0 * P.R * bc.T_w);
        double Uwn = (bc.U_w[0] * n[0] + bc.U_w[1] * n[1]) + bc.U_w[2] * n[2];
        S Uwt[3];
        for (int d = 0; d < 3; ++d) Uwt[d] = bc.U_w[d] - Uwn * n[d];
        S Hw[5], Gw[5];
        half_moments_s(S(Uwn), Uwt, n, lamw, -1, Hw, Gw);
        S rhow = -Gin[0] / (dt * Gw[0]);
        for (int k = 0; k < 5; ++k) F[k] = Gin[k] + dt * rhow * Gw[k];
        return;
    }
    if (bc.type == ORC_BC_SPECULAR) {
        FaceS<S> Rg = L;
        Rg.Un = -L.Un;
        S Ff[5];
        interior_flux_s(L, Rg, false, n, dt, P, Ff);
        S fn = (Ff[1] * n[0] + Ff[2] * n[1]) + Ff[3] * n[2];
        F[0] = 0.0; F[4] = 0.0;
        for (int d = 0; d < 3; ++d) F[1 + d] = fn * n[d];
        return;
    }
    FaceS<S> Rg = (bc.type == ORC_BC_INFLOW) ? face_state_s(bc.W_in, bc.W_in[0], n, P.R) : L;
    Rg.rhoh = Rg.rho;
    interior_flux_s(L, Rg, true, n, dt, P, F);
}

// The parameterised boundary conditions for theta (see the header comment).
template <class S> std::vector<BcS<S>> bcs_of(const orc_params& P, const S theta[3], const std::vector<char>& listed) {
    std::vector<BcS<S>> out(P.n_bc);
    int ff = -1;
    for (int b = 0; b < P.n_bc; ++b)
        if (P.bc[b].type == ORC_BC_INFLOW) { ff = b; break; }
    for (int b = 0; b < P.n_bc; ++b) {
        const orc_bc& c = P.bc[b];
        BcS<S>& o = out[b];
        o.type = c.type;
        o.T_w = c.T_w;
        for (int d = 0; d < 3; ++d) o.U_w[d] = c.U_w[d];
        for (int q = 0; q < 5; ++q) o.W_in[q] = c.W_in[q];
        if (c.type == ORC_BC_DIFFUSE_WALL && listed[b]) o.T_w = theta[2];
        if (c.type == ORC_BC_INFLOW && ff >= 0 && std::memcmp(c.W_in, P.bc[ff].W_in, sizeof(c.W_in)) == 0) {
            const double r0 = c.W_in[0];
            const double U0[3] = {c.W_in[1] / r0, c.W_in[2] / r0, c.W_in[3] / r0};
            const double s0 = std::sqrt((U0[0] * U0[0] + U0[1] * U0[1]) + U0[2] * U0[2]);
            const double e[3] = {s0 > 0.0 ? U0[0] / s0 : 1.0, s0 > 0.0 ? U0[1] / s0 : 0.0, s0 > 0.0 ? U0[2] / s0 : 0.0};
            const double p0 = (c.W_in[4] - 0.5 * r0 * s0 * s0) / 1.5;
            const double RT = p0 / r0;
            o.W_in[0] = theta[0];
            for (int d = 0; d < 3; ++d) o.W_in[1 + d] = theta[0] * theta[1] * e[d];
            o.W_in[4] = theta[0] * (0.5 * theta[1] * theta[1] + 1.5 * RT);
        }
    }
    return out;
}

template <class S> S objective(const SimBase& sim, int K, const double* W0, const double* dtv, const double* rho_p,
                               const double* pflux, const S theta[3], int functional, const std::vector<char>& listed) {
    const Geom& g = sim.g;
    const orc_params& P = sim.P;
    const int nc = g.nc, nf = g.nf;
    const int comp = functional == 0 ? 1 : 4;
    std::vector<BcS<S>> bcs = bcs_of(P, theta, listed);
    std::vector<S> W(5 * (size_t)nc), F(5 * (size_t)nf), rhoh(nc), tau(nc);
    for (size_t k = 0; k < W.size(); ++k) W[k] = W0[k];
    S J = 0.0;
    for (int n = 0; n < K; ++n) {
        const double dt = dtv[n];
        for (int i = 0; i < nc; ++i) {
            S Wi[5];
            for (int q = 0; q < 5; ++q) Wi[q] = W[(size_t)q * nc + i];
            PrimS<S> pr = prim_s(Wi, P.R);
            tau[i] = tau_cell_s(pr, P);
            rhoh[i] = pr.rho - rho_p[(size_t)n * nc + i];
        }
        for (int f = 0; f < nf; ++f) {
            const double* nn = &g.f_n[3 * (size_t)f];
            const int o = g.f_owner[f], nb = g.f_nbr[f];
            S WL[5], Fv[5];
            for (int q = 0; q < 5; ++q) WL[q] = W[(size_t)q * nc + o];
            if (nb >= 0) {
                S WR[5];
                for (int q = 0; q < 5; ++q) WR[q] = W[(size_t)q * nc + nb];
                FaceS<S> L = face_state_s(WL, rhoh[o], nn, P.R), Rs = face_state_s(WR, rhoh[nb], nn, P.R);
                interior_flux_s(L, Rs, false, nn, dt, P, Fv);
            } else {
                boundary_flux_s(WL, rhoh[o], tau[o], bcs[g.f_bc[f]], nn, dt, P, Fv);
                if (listed[g.f_bc[f]]) J = J + Fv[comp] * g.f_area[f];
            }
            for (int q = 0; q < 5; ++q) F[(size_t)q * nf + f] = Fv[q];
        }
        for (int i = 0; i < nc; ++i)
            for (int q = 0; q < 5; ++q) {
                S acc = 0.0;
                for (int k = 0; k < 4; ++k) {
                    const int f = g.tet_face[4 * i + k];
                    S v = F[(size_t)q * nf + f] * g.f_area[f];
                    acc = acc + (g.tet_sign[4 * i + k] > 0 ? v : -v);
                }
                S& Wq = W[(size_t)q * nc + i];
                Wq = (Wq - acc / g.vol[i]) + pflux[((size_t)n * 5 + q) * nc + i] / g.vol[i];
            }
    }
    return J;
}

// Second order: the same map with the limited least-squares reconstruction
// (Sec. 2.1) at the interior faces and first-order boundary faces, as in the
// step, in binary64 only.  The far-field ghosts of the reconstruction hold the
// far-field state at theta.  phi [K][6][nc] holds the limiter values: computed
// and stored with record, taken as given otherwise, so that with phi frozen at
// theta_0 the map is a smooth function of theta whose derivative central
// differences approximate (reading: the limiter is frozen in the derivative).
double objective_o2(const SimBase& sim, int K, const double* W0, const double* dtv, const double* rho_p,
                    const double* pflux, const double theta[3], int functional, const std::vector<char>& listed,
                    double* phi, bool record) {
    const Geom& g = sim.g;
    const int nc = g.nc, nf = g.nf;
    const int comp = functional == 0 ? 1 : 4;
    orc_params Pt = sim.P;
    std::vector<BcS<double>> bcs = bcs_of(sim.P, theta, listed);
    for (int b = 0; b < Pt.n_bc; ++b) {
        Pt.bc[b].T_w = bcs[b].T_w;
        for (int q = 0; q < 5; ++q) Pt.bc[b].W_in[q] = bcs[b].W_in[q];
    }
    std::vector<double> W(W0, W0 + 5 * (size_t)nc), F(5 * (size_t)nf), rhoh(nc), tau(nc), gW, gH;
    double J = 0.0;
    for (int n = 0; n < K; ++n) {
        const double dt = dtv[n];
        for (int i = 0; i < nc; ++i) {
            double Wi[5];
            for (int q = 0; q < 5; ++q) Wi[q] = W[(size_t)q * nc + i];
            Prim pr = prim_of(Wi, Pt.R, 0);
            tau[i] = tau_cell(pr, Pt);
            rhoh[i] = pr.rho - rho_p[(size_t)n * nc + i];
        }
        limited_gradients(g, Pt, W, rhoh, true, gW, gH, phi + (size_t)n * 6 * nc, !record);
        for (int f = 0; f < nf; ++f) {
            const double* nn = &g.f_n[3 * (size_t)f];
            const int o = g.f_owner[f], nb = g.f_nbr[f];
            double WL[5], Fv[5];
            for (int q = 0; q < 5; ++q) WL[q] = W[(size_t)q * nc + o];
            if (nb >= 0) {
                double WR[5], dxL[3], dxR[3];
                for (int q = 0; q < 5; ++q) WR[q] = W[(size_t)q * nc + nb];
                const double* xf = &g.f_c[3 * (size_t)f];
                for (int d = 0; d < 3; ++d) {
                    dxL[d] = xf[d] - g.cen[3 * (size_t)o + d];
                    dxR[d] = xf[d] - g.cen[3 * (size_t)nb + d];
                }
                face_flux_o2(frame_of(nn), WL, rhoh[o], &gW[15 * (size_t)o], &gH[3 * (size_t)o], dxL, WR, rhoh[nb],
                             &gW[15 * (size_t)nb], &gH[3 * (size_t)nb], dxR, dt, false, Pt, Fv);
            } else {
                boundary_flux(WL, rhoh[o], tau[o], Pt.bc[g.f_bc[f]], nn, dt, false, Pt, Fv);
                if (listed[g.f_bc[f]]) J += Fv[comp] * g.f_area[f];
            }
            for (int q = 0; q < 5; ++q) F[(size_t)q * nf + f] = Fv[q];
        }
        for (int i = 0; i < nc; ++i)
            for (int q = 0; q < 5; ++q) {
                double acc = 0.0;
                for (int k = 0; k < 4; ++k) {
                    const int f = g.tet_face[4 * i + k];
                    double v = F[(size_t)q * nf + f] * g.f_area[f];
                    acc += g.tet_sign[4 * i + k] > 0 ? v : -v;
                }
                double& Wq = W[(size_t)q * nc + i];
                Wq = (Wq - acc / g.vol[i]) + pflux[((size_t)n * 5 + q) * nc + i] / g.vol[i];
            }
    }
    return J;
}

}  // namespace frozen

struct orc_sim { SimBase* s; };

static void set_err(char* err, int32_t len, const std::string& msg) {
    if (err && len > 0) { std::snprintf(err, (size_t)len, "%s", msg.c_str()); }
}

extern "C" {

void orc_math_d(int which, const double* x, double* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) {
        double s, c;
        switch (which) {
            case 0: y[k] = exp_d(x[k]); break;
            case 1: y[k] = log_d(x[k]); break;
            case 2: sincos2pi_d(x[k], &s, &c); y[k] = s; break;
            default: sincos2pi_d(x[k], &s, &c); y[k] = c; break;
        }
    }
}

void orc_math_logf(const float* x, float* y, int64_t n) {
    for (int64_t k = 0; k < n; ++k) y[k] = log_f(x[k]);
}

void orc_math_sincos2pi_f(const float* x, float* s, float* c, int64_t n) {
    for (int64_t k = 0; k < n; ++k) sincos2pi_f(x[k], &s[k], &c[k]);
}

void orc_philox32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    Ctr4x32 c;
    for (int k = 0; k < 4; ++k) c.v[k] = ctr[k];
    Ctr4x32 r = philox4x32_10(c, key[0], key[1]);
    for (int k = 0; k < 4; ++k) out[k] = r.v[k];
}

void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    Ctr4 c;
    for (int k = 0; k < 4; ++k) c.v[k] = ctr[k];
    Ctr4 r = philox4x64_10(c, key[0], key[1]);
    for (int k = 0; k < 4; ++k) out[k] = r.v[k];
}

void orc_qcoef(double dt, double tau, double q[7]) { qcoef(dt, tau, q); }

void orc_maxwell_moments(const double U[3], double lam, const double n[3], int half, int32_t K,
                         double H[5], double G[5]) {
    double Un = dot3(U, n), Ut[3];
    for (int d = 0; d < 3; ++d) Ut[d] = U[d] - Un * n[d];
    half_moments(Un, Ut, n, lam, half, K, H, G);
}

int orc_face_flux(const orc_params* p, int kind, const double WL[5], double rhohL,
                  const double WR[5], double rhohR, const double n[3], double dt,
                  double tau_wall, const orc_bc* bc, int32_t gks, double F[5]) {
    if (kind == 0) {
        FaceState L = face_state(WL, rhohL, n, p->R, p->K), R = face_state(WR, rhohR, n, p->R, p->K);
        interior_flux(L, R, false, gks != 0, n, dt, *p, F);
        return 0;
    }
    if (!bc) return -1;
    boundary_flux(WL, rhohL, tau_wall, *bc, n, dt, gks != 0, *p, F);
    return 0;
}

orc_sim* orc_create(const orc_params* p, int32_t n_nodes, const double* xyz,
                    int32_t n_tets, const int32_t* tets, int32_t n_bfaces,
                    const int32_t* bfaces, const int32_t* btags, const double* W0,
                    char* err, int32_t errlen) {
    std::string e;
    if (p->order != 1 && p->order != 2) { set_err(err, errlen, "order must be 1 or 2"); return nullptr; }
    if (p->n_bc < 0 || p->n_bc > 16) { set_err(err, errlen, "n_bc out of range"); return nullptr; }
    if (p->sampling < 0 || p->sampling > 2) { set_err(err, errlen, "unknown sampling mode"); return nullptr; }
    if (p->K < 0 || p->K > 8) { set_err(err, errlen, "K must be in [0, 8]"); return nullptr; }
    if (p->K > 0 && p->sampling != 0) {
        set_err(err, errlen, "internal degrees of freedom (K > 0) need the printed sampling");
        return nullptr;
    }
    if (p->sampling == 2 && p->order != 2) {
        set_err(err, errlen, "first-order g_p sampling needs order 2 (the cell slopes)");
        return nullptr;
    }
    if (n_tets >= (1 << 24)) { set_err(err, errlen, "too many tets for the particle id layout"); return nullptr; }
    SimBase* s = nullptr;
    if (p->precision == ORC_MIXED) s = new Sim<float>(); else s = new Sim<double>();
    s->P = *p;
    if (!build_geometry(s->g, n_nodes, xyz, n_tets, tets, n_bfaces, bfaces, btags, p->n_bc, e)) {
        delete s; set_err(err, errlen, e); return nullptr;
    }
    if (p->precision == ORC_MIXED) static_cast<Sim<float>*>(s)->pl.build(s->g);
    else static_cast<Sim<double>*>(s)->pl.build(s->g);
    s->W.assign(W0, W0 + 5 * (size_t)n_tets);
    scale_exponents(s->g, s->P, s->W, s->e);
    orc_sim* h = new orc_sim;
    h->s = s;
    return h;
}

void orc_free(orc_sim* h) {
    if (!h) return;
    delete h->s;
    delete h;
}

int orc_step(orc_sim* h, char* err, int32_t errlen) {
    std::string e;
    int rc = h->s->do_step(e);
    if (rc) set_err(err, errlen, e);
    return rc;
}

int orc_gks_step(orc_sim* h, int32_t local, char* err, int32_t errlen) {
    std::string e;
    int rc = h->s->gks_step(local != 0, e);
    if (rc) set_err(err, errlen, e);
    return rc;
}

void orc_sizes(const orc_sim* h, int64_t out[5]) {
    out[0] = h->s->g.nc; out[1] = h->s->g.nf; out[2] = h->s->g.nbf;
    out[3] = h->s->n_particles(); out[4] = h->s->step;
}

int orc_geometry(const orc_sim* h, int which, double* out) {
    const Geom& g = h->s->g;
    int nc = g.nc, nf = g.nf;
    switch (which) {
        case 0: for (int i = 0; i < nc; ++i) out[i] = g.vol[i]; return 0;
        case 1: for (int i = 0; i < nc; ++i) for (int d = 0; d < 3; ++d) out[(size_t)d * nc + i] = g.cen[3 * i + d]; return 0;
        case 2: for (int f = 0; f < nf; ++f) for (int d = 0; d < 3; ++d) out[(size_t)d * nf + f] = g.f_n[3 * (size_t)f + d]; return 0;
        case 3: for (int f = 0; f < nf; ++f) out[f] = g.f_area[f]; return 0;
        case 4: for (int f = 0; f < nf; ++f) out[f] = g.f_owner[f]; return 0;
        case 5: for (int f = 0; f < nf; ++f) out[f] = g.f_nbr[f]; return 0;
        case 6: for (int i = 0; i < nc; ++i) for (int d = 0; d < 3; ++d) out[(size_t)d * nc + i] = g.dS[3 * i + d]; return 0;
        case 7: for (int f = 0; f < nf; ++f) out[f] = g.f_d[f]; return 0;
        default: return -1;
    }
}

void orc_get_state(const orc_sim* h, double* W, uint64_t* id, int32_t* cell,
                   double* x, double* u, double* m, int64_t* scal, double* t, double* e) {
    const SimBase* s = h->s;
    if (W) std::memcpy(W, s->W.data(), s->W.size() * sizeof(double));
    s->get_particles(id, cell, x, u, m, e);
    if (scal) { scal[0] = s->step; for (int k = 0; k < 5; ++k) scal[1 + k] = s->e[k]; }
    if (t) *t = s->t;
}

int orc_set_state(orc_sim* h, const double* W, int64_t n, const uint64_t* id,
                  const int32_t* cell, const double* x, const double* u, const double* m,
                  const int64_t* scal, double t, const double* ei, char* err, int32_t errlen) {
    SimBase* s = h->s;
    std::string e;
    if (!s->set_particles(n, id, cell, x, u, m, ei, e)) { set_err(err, errlen, e); return -1; }
    std::memcpy(s->W.data(), W, s->W.size() * sizeof(double));
    s->step = scal[0];
    for (int k = 0; k < 5; ++k) s->e[k] = (int)scal[1 + k];
    s->t = t;
    return 0;
}

int orc_last(const orc_sim* h, int which, void* out) {
    const SimBase* s = h->s;
    switch (which) {
        case 0: *(double*)out = s->dt; return 0;
        case 1: std::memcpy(out, s->tau.data(), s->tau.size() * 8); return 0;
        case 2: std::memcpy(out, s->rhoh.data(), s->rhoh.size() * 8); return 0;
        case 3: std::memcpy(out, s->nsam.data(), s->nsam.size() * 8); return 0;
        case 4: std::memcpy(out, s->msam.data(), s->msam.size() * 8); return 0;
        case 5: std::memcpy(out, s->F.data(), s->F.size() * 8); return 0;
        case 6: std::memcpy(out, s->pflux.data(), s->pflux.size() * 8); return 0;
        case 7: std::memcpy(out, s->smass.data(), s->smass.size() * 8); return 0;
        case 8: std::memcpy(out, s->scount.data(), s->scount.size() * 8); return 0;
        case 9: std::memcpy(out, s->counters, sizeof(s->counters)); return 0;
        default: return -1;
    }
}

int orc_gradients(orc_sim* h, int limited, double* gradW, double* gradH) {
    std::string e;
    SimBase* s = h->s;
    int rc = s->prepare(e);
    if (rc) return rc;
    std::vector<double> gW, gH;
    limited_gradients(s->g, s->P, s->W, s->rhoh, limited != 0, gW, gH);
    const int nc = s->g.nc;
    for (int i = 0; i < nc; ++i) {
        for (int q = 0; q < 5; ++q)
            for (int d = 0; d < 3; ++d) gradW[((size_t)q * 3 + d) * nc + i] = gW[15 * (size_t)i + 3 * q + d];
        for (int d = 0; d < 3; ++d) gradH[(size_t)d * nc + i] = gH[3 * (size_t)i + d];
    }
    return 0;
}

void orc_slope_moment(const double U[3], double lam, int half, int32_t K, const double a[5], int d, double out[5]) {
    FrameMom M = frame_moments(U, lam, half, K);
    for (int k = 0; k < 5; ++k) out[k] = expect(M, mul(mul(mul(coord(0), coord(d)), lin(a)), psi(k)));
}

void orc_micro_slope(const double U[3], double lam, int32_t K, const double b[5], double a[5]) {
    micro_slope(U, lam, K, b, a);
}

int orc_face_flux_o2(const orc_params* p, const double WL[5], double rhohL, const double gWL[15], const double gHL[3],
                     const double dxL[3], const double WR[5], double rhohR, const double gWR[15],
                     const double gHR[3], const double dxR[3], const double n[3], double dt, int32_t gks,
                     double F[5]) {
    Frame R = frame_of(n);
    face_flux_o2(R, WL, rhohL, gWL, gHL, dxL, WR, rhohR, gWR, gHR, dxR, dt, gks != 0, *p, F);
    return 0;
}

int orc_prepare(orc_sim* h, char* err, int32_t errlen) {
    std::string e;
    int rc = h->s->prepare(e);
    if (rc) set_err(err, errlen, e);
    return rc;
}

int64_t orc_sample_cell(const orc_sim* h, int32_t cell, int64_t cap, uint64_t* id, double* x, double* u, double* m,
                        double* e) {
    if (cell < 0 || cell >= h->s->g.nc) return -1;
    return h->s->sample_one_cell(cell, cap, id, x, u, m, e);
}

void orc_gp_draw(int32_t precision, uint64_t seed, uint64_t step, const double coef[14], uint64_t id0, int64_t n,
                 double* X) {
    for (int64_t k = 0; k < n; ++k) {
        if (precision == ORC_MIXED) gp_draw<float>(seed, step, coef, id0 + (uint64_t)k, &X[3 * k]);
        else gp_draw<double>(seed, step, coef, id0 + (uint64_t)k, &X[3 * k]);
    }
}

int orc_gp_coefficients(const orc_sim* h, int32_t cell, double out[14]) {
    if (cell < 0 || cell >= h->s->g.nc) return -1;
    return h->s->gp_coef(cell, out) ? 0 : -1;
}

int orc_track_one(const orc_sim* h, uint64_t id, int32_t cell, double* io_x, double* io_u, double* io_e,
                  double tau_cell_v, double dt, int64_t step, int32_t* cell_out, int32_t* ncross) {
    return h->s->track_one(id, cell, io_x, io_u, io_e, tau_cell_v, dt, step, cell_out, ncross);
}

int orc_frozen_objective(const orc_sim* h, int32_t K, const double* W0, const double* dt, const double* rho_p,
                         const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                         int32_t n_tags, double out[4]) {
    const SimBase& sim = *h->s;
    if (sim.P.order != 1 || sim.P.K != 0 || K < 1 || (functional != 0 && functional != 1)) return -1;
    std::vector<char> listed(16, 0);
    for (int k = 0; k < n_tags; ++k)
        if (tags[k] >= 0 && tags[k] < 16) listed[tags[k]] = 1;
    orc::Dual<3> th[3];
    for (int k = 0; k < 3; ++k) { th[k] = orc::Dual<3>(theta[k]); th[k].d[k] = 1.0; }
    orc::Dual<3> J = frozen::objective(sim, K, W0, dt, rho_p, pflux, th, functional, listed);
    out[0] = J.v;
    for (int k = 0; k < 3; ++k) out[1 + k] = J.d[k];
    return 0;
}

int orc_frozen_value(const orc_sim* h, int32_t K, const double* W0, const double* dt, const double* rho_p,
                     const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                     int32_t n_tags, double* J) {
    const SimBase& sim = *h->s;
    if (sim.P.order != 1 || sim.P.K != 0 || K < 1 || (functional != 0 && functional != 1)) return -1;
    std::vector<char> listed(16, 0);
    for (int k = 0; k < n_tags; ++k)
        if (tags[k] >= 0 && tags[k] < 16) listed[tags[k]] = 1;
    *J = frozen::objective(sim, K, W0, dt, rho_p, pflux, theta, functional, listed);
    return 0;
}

int orc_frozen_o2_value(const orc_sim* h, int32_t K, const double* W0, const double* dt, const double* rho_p,
                        const double* pflux, const double theta[3], int32_t functional, const int32_t* tags,
                        int32_t n_tags, double* phi, int32_t record, double* J) {
    const SimBase& sim = *h->s;
    if (sim.P.order != 2 || sim.P.K != 0 || K < 1 || (functional != 0 && functional != 1)) return -1;
    std::vector<char> listed(16, 0);
    for (int k = 0; k < n_tags; ++k)
        if (tags[k] >= 0 && tags[k] < 16) listed[tags[k]] = 1;
    *J = frozen::objective_o2(sim, K, W0, dt, rho_p, pflux, theta, functional, listed, phi, record != 0);
    return 0;
}

}  // extern "C"
