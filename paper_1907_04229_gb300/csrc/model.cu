// The step either side of the linear solve: the fully implicit residual, its analytic Jacobian and the
// discrete Schur approximation S_e of the thermal multiphase finite-volume model, assembled on the
// device, and Newton's method with a backtracking line search for one implicit Euler step (Sec. 3
// eq. (AXR): each Newton iteration solves J dx = -R with CPTR-FGMRES; Sec. 4: Newton with line
// search, relative function-norm and step-norm tolerances).
//
// Model (Sec. 2): phase mass conservation with Darcy flow (capillarity ignored) and the energy
// equation with advection and conduction; S_o eliminated by the saturation constraint; unknowns per
// cell (p, T, S_w[, S_g]); raw equation rows water mass, energy, oil mass[, gas mass].  Discretised
// by TPFA on a Cartesian box (harmonic K and k_T, arithmetic face density, phase upwinding on the
// potential difference with ties to the lower-index cell) and implicit Euler (Sec. 2.2).  Water
// density and viscosity follow Appendix A (Kell / Grabowski correlations as printed).  The laws the
// paper leaves to its companion paper are parameters: oil density exp(c_o (p - p0) - beta_o (T - T0)),
// oil viscosity mu_ref exp(-beta_mu (T - T0)), ideal gas, Corey k_r = S^n, producers
// q_alpha = WI lam_alpha (p - p_bh)^+, injectors of water at a fixed rate and temperature, heaters
// U (T_heater - T).  S_e (eq. Se) is the energy equation with every coefficient frozen at the
// current iterate, differentiated in the explicit temperature factors only.
//
// Layout: one thread per cell gathers its own rows: the cell's accumulation terms, its wells and
// heaters (in the caller's order), then its six faces in the order (i - nx ny, i), (i - nx, i),
// (i - 1, i), (i, i + 1), (i, i + nx), (i, i + nx ny).  Each face is evaluated by both of its cells
// with the same operations, so the two rows see the same flux.  This file is compiled without
// fused multiply-adds: every product and sum is rounded on its own.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

namespace cptr {

namespace {

constexpr int kMaxB = 4;
constexpr double kRgas = 8.314462618;

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// scalar parameters and device arrays of the model (passed by value to the kernels)
struct DevModel {
    int32_t nx, ny, nz, nphase, b, n_wells, n_heaters, pad;
    double dx, dy, dz, dt, phi, grav;
    double kT_const, kT_rock, kT_w, kT_o, kT_g;
    double cv_w, cv_o, cv_g, c_rock, rho_rock;
    double mu_o_ref, beta_mu, T0, rho_o_ref, c_o, beta_o, p0;
    double gas_M, mu_g, corey_n;
    const double *kh, *kv;
    const int32_t *src_ptr, *src_idx;   // per cell: wells w >= 0 and heaters -(h + 1), in the caller's order
    const int32_t *well_kind;
    const double *well_a, *well_c, *heater_U, *heater_T;
};

struct Phase {
    double S, dS[kMaxB], rho, drho[kMaxB], lam, dlam[kMaxB], rl, drl[kMaxB];
};
struct CellState {
    Phase ph[3];
    double kT, dkT[kMaxB];
};

__device__ __forceinline__ int raw_row(int a) { return a == 0 ? 0 : (a == 1 ? 2 : 3); }
__device__ __forceinline__ double cv_of(const DevModel &m, int a) { return a == 0 ? m.cv_w : (a == 1 ? m.cv_o : m.cv_g); }
__device__ __forceinline__ double harm(double a, double b) { return 2.0 * a * b / (a + b); }

// water density (Kell's fit times the pressure factor) and viscosity (Grabowski), Appendix A
__device__ void water_props(double p, double T, double *rho, double *rp, double *rT, double *mu, double *mT) {
    const double E0 = 999.83952, E1 = 16.955176, E2 = -7.987e-3, E3 = -46.170461e-6, E4 = 105.56302e-9,
                 E5 = -280.54353e-12, E6 = 16.87985e-3, E7 = 10.2, Cw = 3.98854e-4;
    const double A = 2.1850, B = 0.04012, C = 5.1547e-6;
    const double Tc = T - 273.15;
    const double poly = E0 + Tc * (E1 + Tc * (E2 + Tc * (E3 + Tc * (E4 + Tc * E5))));
    const double dpoly = E1 + Tc * (2 * E2 + Tc * (3 * E3 + Tc * (4 * E4 + Tc * 5 * E5)));
    const double den = 1.0 + E6 * Tc;
    const double f = poly / den, df = (dpoly * den - poly * E6) / (den * den);
    const double ex = exp(Cw * (p * 1e-6 - E7));
    *rho = f * ex;
    *rp = *rho * Cw * 1e-6;
    *rT = df * ex;
    const double TF = Tc * 1.8 + 32.0;
    const double q = -1.0 + B * TF + C * TF * TF;
    *mu = 1e-3 * A / q;
    *mT = -1e-3 * A * (B + 2.0 * C * TF) * 1.8 / (q * q);
}

// saturations, densities, mobilities and conductivity of one cell, with their derivatives
__device__ void cell_eval(const DevModel &m, const double *u, CellState *cs) {
    const int b = m.b;
    const double p = u[0], T = u[1], Sw = u[2], Sg = m.nphase == 3 ? u[3] : 0.0;
    for (int a = 0; a < 3; ++a) {
        Phase &s = cs->ph[a];
        s.S = s.rho = s.lam = s.rl = 0.0;
        for (int c = 0; c < kMaxB; ++c) s.dS[c] = s.drho[c] = s.dlam[c] = s.drl[c] = 0.0;
    }
    cs->kT = 0.0;
    for (int c = 0; c < kMaxB; ++c) cs->dkT[c] = 0.0;
    for (int a = 0; a < m.nphase; ++a) {
        Phase &s = cs->ph[a];
        double rho, rp, rT, mu, mT;
        if (a == 0) {
            water_props(p, T, &rho, &rp, &rT, &mu, &mT);
            s.S = Sw;
            s.dS[2] = 1.0;
        } else if (a == 1) {
            rho = m.rho_o_ref * exp(m.c_o * (p - m.p0) - m.beta_o * (T - m.T0));
            rp = m.c_o * rho;
            rT = -m.beta_o * rho;
            mu = m.mu_o_ref * exp(-m.beta_mu * (T - m.T0));
            mT = -m.beta_mu * mu;
            s.S = 1.0 - Sw - Sg;
            s.dS[2] = -1.0;
            if (b == 4) s.dS[3] = -1.0;
        } else {
            rho = p * m.gas_M / (kRgas * T);
            rp = m.gas_M / (kRgas * T);
            rT = -rho / T;
            mu = m.mu_g;
            mT = 0.0;
            s.S = Sg;
            s.dS[3] = 1.0;
        }
        s.rho = rho;
        s.drho[0] = rp;
        s.drho[1] = rT;
        const double Sc = s.S > 0.0 ? s.S : 0.0;
        const double kr = pow(Sc, m.corey_n);
        const double dkr = s.S > 0.0 ? m.corey_n * pow(Sc, m.corey_n - 1.0) : 0.0;
        s.lam = kr / mu;
        for (int c = 0; c < b; ++c) s.dlam[c] = dkr * s.dS[c] / mu;
        s.dlam[1] += -kr * mT / (mu * mu);
        s.rl = rho * s.lam;
        for (int c = 0; c < b; ++c) s.drl[c] = s.drho[c] * s.lam + rho * s.dlam[c];
    }
    if (m.kT_const > 0.0) {
        cs->kT = m.kT_const;
    } else {
        const double kf[3] = {m.kT_w, m.kT_o, m.kT_g};
        cs->kT = (1.0 - m.phi) * m.kT_rock;
        for (int a = 0; a < m.nphase; ++a) {
            cs->kT += m.phi * cs->ph[a].S * kf[a];
            for (int c = 0; c < b; ++c) cs->dkT[c] += m.phi * kf[a] * cs->ph[a].dS[c];
        }
    }
}

// position of column j in row i (rows sorted), -1 if absent
__device__ __forceinline__ int32_t find_col(const int32_t *rp, const int32_t *ci, int32_t i, int32_t j) {
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == j) return k;
    return -1;
}

// One thread per cell i: its raw residual rows R_i, its block row of J (if J) and its row of S_e (if
// Se), on the 7-point pattern (rp, ci).  err is set if the pattern lacks a block the model needs.
template <int B>
__global__ void k_assemble(DevModel m, const double *__restrict__ x, const double *__restrict__ xn,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, double *R, double *J,
                           double *Se, int32_t *err) {
    constexpr int BB = B * B;
    const int64_t n = (int64_t)m.nx * m.ny * m.nz;
    const int64_t ii = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ii >= n) return;
    const int32_t i = (int32_t)ii, nxy = m.nx * m.ny;
    const int np = m.nphase;
    const double V = m.dx * m.dy * m.dz;
    double Ri[B];
    for (int r = 0; r < B; ++r) Ri[r] = 0.0;
    if (J)
        for (int64_t e = (int64_t)rp[i] * BB; e < (int64_t)rp[i + 1] * BB; ++e) J[e] = 0.0;
    if (Se)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) Se[k] = 0.0;
    const int32_t kd = find_col(rp, ci, i, i);
    if (kd < 0) { atomicExch(err, 1); return; }
    double *Jd = J ? J + (int64_t)kd * BB : nullptr;
    // accumulation: V (phi rho S - (phi rho S)^n) / dt per phase; energy with rock heat
    {
        CellState cs, cn;
        const double *u = x + ii * B, *un = xn + ii * B;
        cell_eval(m, u, &cs);
        cell_eval(m, un, &cn);
        const double T = u[1], Tn = un[1];
        const double acc = V / m.dt;
        double eacc = 0.0;
        for (int a = 0; a < np; ++a) {
            const Phase &s = cs.ph[a], &sn = cn.ph[a];
            const double cv = cv_of(m, a);
            Ri[raw_row(a)] += acc * m.phi * (s.rho * s.S - sn.rho * sn.S);
            eacc += m.phi * cv * (s.rho * s.S * T - sn.rho * sn.S * Tn);
            if (Jd)
                for (int c = 0; c < B; ++c) {
                    const double dm = s.drho[c] * s.S + s.rho * s.dS[c];
                    Jd[raw_row(a) * B + c] += acc * m.phi * dm;
                    Jd[1 * B + c] += acc * m.phi * cv * (dm * T + (c == 1 ? s.rho * s.S : 0.0));
                }
            if (Se) Se[kd] += acc * m.phi * cv * s.S * s.rho;
        }
        eacc += (1.0 - m.phi) * m.rho_rock * m.c_rock * (T - Tn);
        Ri[1] += acc * eacc;
        if (Jd) Jd[1 * B + 1] += acc * (1.0 - m.phi) * m.rho_rock * m.c_rock;
        if (Se) Se[kd] += acc * (1.0 - m.phi) * m.rho_rock * m.c_rock;
    }
    // wells and heaters of this cell, in the caller's order (wells first)
    for (int32_t q = m.src_ptr[i]; q < m.src_ptr[i + 1]; ++q) {
        const int32_t w = m.src_idx[q];
        const double *u = x + ii * B;
        if (w < 0) {   // heater U (T_heater - T)
            const int32_t h = -w - 1;
            const double U = m.heater_U[h];
            Ri[1] -= U * (m.heater_T[h] - u[1]);
            if (Jd) Jd[1 * B + 1] += U;
            if (Se) Se[kd] += U;
        } else if (m.well_kind[w] == 0) {   // injector: water at T_inj, mass source q rho_w(p, T_inj)
            const double qv = m.well_a[w], Tinj = m.well_c[w];
            double rho, rp_, rT, mu, mT;
            water_props(u[0], Tinj, &rho, &rp_, &rT, &mu, &mT);
            Ri[0] -= qv * rho;
            Ri[1] -= m.cv_w * Tinj * qv * rho;
            if (Jd) {
                Jd[0 * B + 0] -= qv * rp_;
                Jd[1 * B + 0] -= m.cv_w * Tinj * qv * rp_;
            }
        } else {   // producer: q_alpha = WI lam_alpha (p - p_bh)^+, mass sink rho_alpha q_alpha
            const double WI = m.well_a[w], dp = u[0] - m.well_c[w];
            if (dp <= 0.0) continue;
            CellState cs;
            cell_eval(m, u, &cs);
            const double T = u[1];
            for (int a = 0; a < np; ++a) {
                const Phase &s = cs.ph[a];
                const double cv = cv_of(m, a);
                const double mm = WI * s.rl * dp;
                Ri[raw_row(a)] += mm;
                Ri[1] += cv * T * mm;
                if (Jd)
                    for (int c = 0; c < B; ++c) {
                        const double dm = WI * dp * s.drl[c] + (c == 0 ? WI * s.rl : 0.0);
                        Jd[raw_row(a) * B + c] += dm;
                        Jd[1 * B + c] += cv * (T * dm + (c == 1 ? mm : 0.0));
                    }
                if (Se) Se[kd] += cv * mm;
            }
        }
    }
    // the six faces: i as the upper cell of (i - nxy, i), (i - nx, i), (i - 1, i), then as the lower
    // cell of (i, i + 1), (i, i + nx), (i, i + nxy)
    const int32_t x0 = i % m.nx, y0 = (i / m.nx) % m.ny, z0 = i / nxy;
    for (int f = 0; f < 6; ++f) {
        const bool low = f >= 3;           // i is the face's lower-index cell L
        const int dir = low ? f - 3 : 2 - f;
        int32_t L, Rc;
        double area, dist, dzLR;
        if (dir == 0) {
            if (low ? x0 == m.nx - 1 : x0 == 0) continue;
            L = low ? i : i - 1;
            area = m.dy * m.dz; dist = m.dx; dzLR = 0.0;
            Rc = L + 1;
        } else if (dir == 1) {
            if (low ? y0 == m.ny - 1 : y0 == 0) continue;
            L = low ? i : i - m.nx;
            area = m.dx * m.dz; dist = m.dy; dzLR = 0.0;
            Rc = L + m.nx;
        } else {
            if (low ? z0 == m.nz - 1 : z0 == 0) continue;
            L = low ? i : i - nxy;
            area = m.dx * m.dy; dist = m.dz; dzLR = -m.dz;   // depth grows with z
            Rc = L + nxy;
        }
        const double KL = dir == 2 ? m.kv[L] : m.kh[L], KR = dir == 2 ? m.kv[Rc] : m.kh[Rc];
        const double *uL = x + (int64_t)L * B, *uR = x + (int64_t)Rc * B;
        CellState sL, sR;
        cell_eval(m, uL, &sL);
        cell_eval(m, uR, &sR);
        const double Ups = area / dist * harm(KL, KR);
        const int32_t other = low ? Rc : L;
        const int32_t ko = find_col(rp, ci, i, other);   // block (i, other)
        if (ko < 0) { atomicExch(err, 1); return; }
        // the row's own blocks: (L, L), (L, R) seen from L; (R, L), (R, R) seen from R
        const int32_t kLx = low ? kd : ko, kRx = low ? ko : kd;   // block of column L / column R in row i
        const double sg = low ? 1.0 : -1.0;
        for (int a = 0; a < np; ++a) {
            const Phase &pL = sL.ph[a], &pR = sR.ph[a];
            const double cv = cv_of(m, a);
            const double rbar = 0.5 * (pL.rho + pR.rho);
            const double Phi = (uL[0] - uR[0]) - rbar * m.grav * dzLR;
            const bool upL = Phi >= 0.0;   // tie: the lower-index cell
            const Phase &pu = upL ? pL : pR;
            const double Tup = upL ? uL[1] : uR[1];
            const double F = Ups * pu.rl * Phi;
            const int ra = raw_row(a);
            if (low) {
                Ri[ra] += F;
                Ri[1] += cv * Tup * F;
            } else {
                Ri[ra] -= F;
                Ri[1] -= cv * Tup * F;
            }
            if (J) {
                double dFL[B], dFR[B];
                for (int c = 0; c < B; ++c) {
                    const double dPhiL = (c == 0 ? 1.0 : 0.0) - 0.5 * pL.drho[c] * m.grav * dzLR;
                    const double dPhiR = (c == 0 ? -1.0 : 0.0) - 0.5 * pR.drho[c] * m.grav * dzLR;
                    dFL[c] = Ups * (pu.rl * dPhiL + (upL ? Phi * pL.drl[c] : 0.0));
                    dFR[c] = Ups * (pu.rl * dPhiR + (upL ? 0.0 : Phi * pR.drl[c]));
                }
                double *JL = J + (int64_t)kLx * BB, *JR = J + (int64_t)kRx * BB;
                for (int c = 0; c < B; ++c) {
                    const double dGL = cv * (Tup * dFL[c] + ((upL && c == 1) ? F : 0.0));
                    const double dGR = cv * (Tup * dFR[c] + ((!upL && c == 1) ? F : 0.0));
                    if (low) {
                        JL[ra * B + c] += dFL[c];
                        JR[ra * B + c] += dFR[c];
                        JL[1 * B + c] += dGL;
                        JR[1 * B + c] += dGR;
                    } else {
                        JL[ra * B + c] -= dFL[c];
                        JR[ra * B + c] -= dFR[c];
                        JL[1 * B + c] -= dGL;
                        JR[1 * B + c] -= dGR;
                    }
                }
            }
            if (Se) {   // the frozen mass flux advects delta T from the upwind cell
                const int32_t ku = upL ? kLx : kRx;
                Se[ku] += sg * (cv * F);
            }
        }
        // conduction with harmonic k_T
        const double khT = harm(sL.kT, sR.kT);
        const double UT = area / dist * khT;
        const double dT = uL[1] - uR[1];
        if (low) Ri[1] += UT * dT;
        else Ri[1] -= UT * dT;
        if (J) {
            const double s2 = (sL.kT + sR.kT) * (sL.kT + sR.kT);
            const double dhL = 2.0 * sR.kT * sR.kT / s2, dhR = 2.0 * sL.kT * sL.kT / s2;
            double *JL = J + (int64_t)kLx * BB, *JR = J + (int64_t)kRx * BB;
            for (int c = 0; c < B; ++c) {
                const double gL = area / dist * dhL * sL.dkT[c] * dT + (c == 1 ? UT : 0.0);
                const double gR = area / dist * dhR * sR.dkT[c] * dT - (c == 1 ? UT : 0.0);
                if (low) {
                    JL[1 * B + c] += gL;
                    JR[1 * B + c] += gR;
                } else {
                    JL[1 * B + c] -= gL;
                    JR[1 * B + c] -= gR;
                }
            }
        }
        if (Se) {
            if (low) { Se[kd] += UT; Se[ko] -= UT; }
            else { Se[kd] += UT; Se[ko] -= UT; }
        }
    }
    for (int r = 0; r < B; ++r) R[ii * B + r] = Ri[r];
}

// ------------------------------------------------------------------------------------------------
// vector kernels of the Newton loop
__global__ void k_neg(int64_t n, const double *a, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = -a[i];
}
__global__ void k_axpy_to(int64_t n, const double *x, double alpha, const double *d, double *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i] + alpha * d[i];
}
// sum of squares of (W R) per block of 256 cells' entries: partial[blockIdx] (fixed order), W per cell
// b x b row-major (null: identity)
template <int B>
__global__ void __launch_bounds__(256) k_wnorm_partial(int32_t n, const double *W, const double *R, double *partial) {
    __shared__ double sh[256];
    const int32_t i = blockIdx.x * 256 + threadIdx.x;
    double s = 0.0;
    if (i < n)
        for (int r = 0; r < B; ++r) {
            double v = 0.0;
            if (W)
                for (int t = 0; t < B; ++t) v += W[((int64_t)i * B + r) * B + t] * R[(int64_t)i * B + t];
            else
                v = R[(int64_t)i * B + r];
            s += v * v;
        }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
__global__ void __launch_bounds__(256) k_sumsq_partial(int64_t n, const double *a, double *partial) {
    __shared__ double sh[256];
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const double v = i < n ? a[i] : 0.0;
    sh[threadIdx.x] = v * v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}
// the partials summed in block order by one thread: out = sqrt(sum)
__global__ void k_sum_sqrt(int32_t nparts, const double *partial, double *out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int32_t k = 0; k < nparts; ++k) s += partial[k];
        *out = sqrt(s);
    }
}

// the context's model: device copies and the per-cell source lists
struct Model {
    DevModel dm{};
    double *kh = nullptr, *kv = nullptr, *well_a = nullptr, *well_c = nullptr, *heater_U = nullptr,
           *heater_T = nullptr, *W = nullptr;
    int32_t *src_ptr = nullptr, *src_idx = nullptr, *well_kind = nullptr;
    int32_t *rp = nullptr, *ci = nullptr, *kind = nullptr;   // the 7-point pattern, unknown kinds
    int32_t n = 0, nnzb = 0;
};

void model_release(Model *m) {
    if (!m) return;
    for (void *p : {(void *)m->kh, (void *)m->kv, (void *)m->well_a, (void *)m->well_c, (void *)m->heater_U,
                    (void *)m->heater_T, (void *)m->W, (void *)m->src_ptr, (void *)m->src_idx, (void *)m->well_kind,
                    (void *)m->rp, (void *)m->ci, (void *)m->kind})
        dfree(p);
    delete m;
}

template <typename T>
cptr_status to_device(Ctx *c, T **dst, const T *src, size_t count, int on_device) {
    CPTR_TRY(dalloc_t(c, dst, std::max<size_t>(count, 1)));
    if (count)
        CPTR_CUDA_TRY(c, cudaMemcpyAsync(*dst, src, sizeof(T) * count,
                                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    return CPTR_OK;
}
template <typename T>
cptr_status to_host(Ctx *c, std::vector<T> &dst, const T *src, size_t count, int on_device) {
    dst.resize(count);
    if (!count) return CPTR_OK;
    if (on_device) return copy_to_host(c, dst.data(), src, sizeof(T) * count);
    std::copy(src, src + count, dst.begin());
    return CPTR_OK;
}

cptr_status model_set(Ctx *c, const cptr_model *pm, int on_device) {
    if (!pm || pm->nx < 1 || pm->ny < 1 || pm->nz < 1 || (pm->nphase != 2 && pm->nphase != 3) || !pm->kh ||
        !pm->kv || pm->n_wells < 0 || pm->n_heaters < 0 || !(pm->dt > 0.0))
        return c->fail(CPTR_EINVAL, "cptr_model_set: bad model description");
    const int64_t n64 = (int64_t)pm->nx * pm->ny * pm->nz;
    if (n64 > INT32_MAX / 8) return c->fail(CPTR_EINVAL, "cptr_model_set: grid too large");
    const int32_t n = (int32_t)n64, b = pm->nphase + 1;
    Model *m = new (std::nothrow) Model();
    if (!m) return c->fail(CPTR_ENOMEM, "host allocation failed");
    model_release(static_cast<Model *>(c->model));
    c->model = m;
    m->n = n;
    DevModel &d = m->dm;
    d.nx = pm->nx; d.ny = pm->ny; d.nz = pm->nz; d.nphase = pm->nphase; d.b = b;
    d.dx = pm->dx; d.dy = pm->dy; d.dz = pm->dz; d.dt = pm->dt; d.phi = pm->phi; d.grav = pm->grav;
    d.kT_const = pm->kT_const; d.kT_rock = pm->kT_rock; d.kT_w = pm->kT_w; d.kT_o = pm->kT_o; d.kT_g = pm->kT_g;
    d.cv_w = pm->cv_w; d.cv_o = pm->cv_o; d.cv_g = pm->cv_g; d.c_rock = pm->c_rock; d.rho_rock = pm->rho_rock;
    d.mu_o_ref = pm->mu_o_ref; d.beta_mu = pm->beta_mu; d.T0 = pm->T0; d.rho_o_ref = pm->rho_o_ref;
    d.c_o = pm->c_o; d.beta_o = pm->beta_o; d.p0 = pm->p0; d.gas_M = pm->gas_M; d.mu_g = pm->mu_g;
    d.corey_n = pm->corey_n;
    d.n_wells = pm->n_wells;
    d.n_heaters = pm->n_heaters;
    CPTR_TRY(to_device(c, &m->kh, pm->kh, (size_t)n, on_device));
    CPTR_TRY(to_device(c, &m->kv, pm->kv, (size_t)n, on_device));
    // wells and heaters: per-cell lists in the caller's order (wells first), built on the host
    std::vector<int32_t> wc, wk, hc;
    std::vector<double> wa, wcv, hU, hT;
    CPTR_TRY(to_host(c, wc, pm->well_cell, (size_t)pm->n_wells, on_device));
    CPTR_TRY(to_host(c, wk, pm->well_kind, (size_t)pm->n_wells, on_device));
    CPTR_TRY(to_host(c, wa, pm->well_a, (size_t)pm->n_wells, on_device));
    CPTR_TRY(to_host(c, wcv, pm->well_c, (size_t)pm->n_wells, on_device));
    CPTR_TRY(to_host(c, hc, pm->heater_cell, (size_t)pm->n_heaters, on_device));
    CPTR_TRY(to_host(c, hU, pm->heater_U, (size_t)pm->n_heaters, on_device));
    CPTR_TRY(to_host(c, hT, pm->heater_T, (size_t)pm->n_heaters, on_device));
    std::vector<int32_t> sp((size_t)n + 1, 0), si;
    for (int32_t w : wc) {
        if (w < 0 || w >= n) return c->fail(CPTR_EINVAL, "cptr_model_set: well cell out of range");
        ++sp[w + 1];
    }
    for (int32_t h : hc) {
        if (h < 0 || h >= n) return c->fail(CPTR_EINVAL, "cptr_model_set: heater cell out of range");
        ++sp[h + 1];
    }
    for (int32_t i = 0; i < n; ++i) sp[i + 1] += sp[i];
    si.resize(sp[n]);
    std::vector<int32_t> fill(sp.begin(), sp.end() - 1);
    for (int32_t w = 0; w < pm->n_wells; ++w) si[fill[wc[w]]++] = w;
    for (int32_t h = 0; h < pm->n_heaters; ++h) si[fill[hc[h]]++] = -(h + 1);
    CPTR_TRY(to_device(c, &m->src_ptr, sp.data(), sp.size(), 0));
    CPTR_TRY(to_device(c, &m->src_idx, si.data(), si.size(), 0));
    CPTR_TRY(to_device(c, &m->well_kind, wk.data(), wk.size(), 0));
    CPTR_TRY(to_device(c, &m->well_a, wa.data(), wa.size(), 0));
    CPTR_TRY(to_device(c, &m->well_c, wcv.data(), wcv.size(), 0));
    CPTR_TRY(to_device(c, &m->heater_U, hU.data(), hU.size(), 0));
    CPTR_TRY(to_device(c, &m->heater_T, hT.data(), hT.size(), 0));
    if (pm->weights) CPTR_TRY(to_device(c, &m->W, pm->weights, (size_t)n * b * b, on_device));
    // the 7-point pattern in natural order, columns ascending
    std::vector<int32_t> rp((size_t)n + 1, 0), ci;
    const int32_t nx = pm->nx, ny = pm->ny, nz = pm->nz, nxy = nx * ny;
    ci.reserve((size_t)n * 7);
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t xx = 0; xx < nx; ++xx) {
                const int32_t i = xx + nx * (y + ny * z);
                if (z > 0) ci.push_back(i - nxy);
                if (y > 0) ci.push_back(i - nx);
                if (xx > 0) ci.push_back(i - 1);
                ci.push_back(i);
                if (xx < nx - 1) ci.push_back(i + 1);
                if (y < ny - 1) ci.push_back(i + nx);
                if (z < nz - 1) ci.push_back(i + nxy);
                rp[i + 1] = (int32_t)ci.size();
            }
    m->nnzb = rp[n];
    CPTR_TRY(to_device(c, &m->rp, rp.data(), rp.size(), 0));
    CPTR_TRY(to_device(c, &m->ci, ci.data(), ci.size(), 0));
    std::vector<int32_t> kind = {CPTR_U_P, CPTR_U_T, CPTR_U_SAT, CPTR_U_SAT};
    CPTR_TRY(to_device(c, &m->kind, kind.data(), (size_t)b, 0));
    d.kh = m->kh; d.kv = m->kv; d.src_ptr = m->src_ptr; d.src_idx = m->src_idx; d.well_kind = m->well_kind;
    d.well_a = m->well_a; d.well_c = m->well_c; d.heater_U = m->heater_U; d.heater_T = m->heater_T;
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the host vectors are freed on return
    return CPTR_OK;
}

cptr_status assemble(Ctx *c, const double *x, const double *xn, double *R, double *J, double *Se) {
    Model *m = static_cast<Model *>(c->model);
    CPTR_CUDA_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int32_t), c->stream));
    if (m->dm.b == 3)
        (k_assemble<3><<<nblk(m->n, 128), 128, 0, c->stream>>>(m->dm, x, xn, m->rp, m->ci, R, J, Se, c->flag),
         note_launch());
    else
        (k_assemble<4><<<nblk(m->n, 128), 128, 0, c->stream>>>(m->dm, x, xn, m->rp, m->ci, R, J, Se, c->flag),
         note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return CPTR_OK;
}

// ||W R||_2 or ||a||_2 into the host (deterministic: block partials summed in block order)
cptr_status norm2(Ctx *c, const double *R, const double *W, bool weighted, int64_t len, double *partial,
                  double *dout, double *out) {
    Model *m = static_cast<Model *>(c->model);
    int32_t nparts;
    if (weighted) {
        nparts = (int32_t)nblk(m->n, 256);
        if (m->dm.b == 3) (k_wnorm_partial<3><<<nparts, 256, 0, c->stream>>>(m->n, W, R, partial), note_launch());
        else (k_wnorm_partial<4><<<nparts, 256, 0, c->stream>>>(m->n, W, R, partial), note_launch());
    } else {
        nparts = (int32_t)nblk(len, 256);
        (k_sumsq_partial<<<nparts, 256, 0, c->stream>>>(len, R, partial), note_launch());
    }
    (k_sum_sqrt<<<1, 32, 0, c->stream>>>(nparts, partial, dout), note_launch());
    CPTR_CUDA_TRY(c, cudaGetLastError());
    return copy_to_host(c, out, dout, sizeof(double));
}

cptr_status newton(cptr_ctx *ctx, Ctx *c, double *xio, const double *xn_in, double rtol_lin, int32_t max_newton,
                   cptr_newton_stats *st, int on_device) {
    Model *m = static_cast<Model *>(c->model);
    const int b = m->dm.b;
    const int64_t nb = (int64_t)m->n * b;
    cudaStream_t s = c->stream;
    double *x = nullptr, *xn = nullptr, *xt = nullptr, *R = nullptr, *mR = nullptr, *dx = nullptr, *J = nullptr,
           *Se = nullptr, *partial = nullptr, *dnorm = nullptr;
    struct Bufs {
        std::vector<void *> p;
        ~Bufs() { for (void *q : p) dfree(q); }
    } keep;
    auto alloc = [&](double **p, size_t cnt) -> cptr_status {
        CPTR_TRY(dalloc_t(c, p, std::max<size_t>(cnt, 1)));
        keep.p.push_back(*p);
        return CPTR_OK;
    };
    for (double **p : {&x, &xn, &xt, &R, &mR, &dx}) CPTR_TRY(alloc(p, (size_t)nb));
    CPTR_TRY(alloc(&J, (size_t)m->nnzb * b * b));
    CPTR_TRY(alloc(&Se, (size_t)m->nnzb));
    CPTR_TRY(alloc(&partial, (size_t)nblk(nb, 256) + 8));
    CPTR_TRY(alloc(&dnorm, 1));
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(x, xio, sizeof(double) * nb, kin, s));
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(xn, xn_in, sizeof(double) * nb, kin, s));
    cptr_newton_stats out{};
    auto check_pattern = [&]() -> cptr_status {
        int32_t e = 0;
        CPTR_TRY(copy_to_host(c, &e, c->flag, sizeof(int32_t)));
        if (e) return c->fail(CPTR_EINVAL, "model assembly: pattern lacks a block");
        return CPTR_OK;
    };
    // F(x) = ||W R(x)||; Newton until F <= 1e-8 F(x^0) or the relative step ||a dx|| / ||x|| <= 1e-8
    CPTR_TRY(assemble(c, x, xn, R, nullptr, nullptr));
    CPTR_TRY(check_pattern());
    double F0 = 0.0;
    CPTR_TRY(norm2(c, R, m->W, true, nb, partial, dnorm, &F0));
    out.res0 = F0;
    double F = F0;
    const double kTol = 1e-8;
    int it = 0;
    for (; it < max_newton; ++it) {
        if (!(F > kTol * F0) || F == 0.0) { out.converged = 1; break; }
        CPTR_TRY(assemble(c, x, xn, R, J, Se));
        (k_neg<<<nblk(nb, 256), 256, 0, s>>>(nb, R, mR), note_launch());
        // the linear step with CPTR-FGMRES (set-up on this Jacobian, its S_e, the model's weights)
        cptr_status rc = cptr_setup(ctx, m->n, b, m->rp, m->ci, J, m->kind, m->W, Se, 1);
        if (rc != CPTR_OK) return rc;
        cptr_stats ls{};
        rc = cptr_solve(ctx, mR, dx, rtol_lin, &ls, 1);
        if (rc != CPTR_OK && rc != CPTR_NOT_CONVERGED) return rc;
        out.linear_its += ls.iters;
        out.setup_ms += ls.setup_ms;
        out.solve_ms += ls.solve_ms;
        // backtracking line search on F: a = 1, 1/2, ... until F(x + a dx) <= (1 - 1e-4 a) F
        double a = 1.0, Ft = 0.0;
        int cut = 0;
        for (;;) {
            (k_axpy_to<<<nblk(nb, 256), 256, 0, s>>>(nb, x, a, dx, xt), note_launch());
            CPTR_TRY(assemble(c, xt, xn, R, nullptr, nullptr));
            CPTR_TRY(norm2(c, R, m->W, true, nb, partial, dnorm, &Ft));
            if (Ft <= (1.0 - 1e-4 * a) * F || cut >= 10) break;
            a *= 0.5;
            ++cut;
        }
        out.line_search_cuts += cut;
        double dxn = 0.0, xnrm = 0.0;
        CPTR_TRY(norm2(c, dx, nullptr, false, nb, partial, dnorm, &dxn));
        CPTR_TRY(norm2(c, x, nullptr, false, nb, partial, dnorm, &xnrm));
        std::swap(x, xt);
        F = Ft;
        out.newton_its = it + 1;
        if (a * dxn <= kTol * xnrm) { out.converged = F <= F0 ? 1 : 0; ++it; break; }
    }
    if (!out.converged && !(F > kTol * F0)) out.converged = 1;
    out.res = F;
    CPTR_CUDA_TRY(c, cudaMemcpyAsync(xio, x, sizeof(double) * nb,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CPTR_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (st) *st = out;
    return out.converged ? CPTR_OK : CPTR_NOT_CONVERGED;
}

template <typename Fn>
cptr_status guard(cptr_ctx *ctx, Fn &&f) {
    if (!ctx) return CPTR_EINVAL;
    Ctx *c = &ctx->c;
    CtxScope scope(c);
    try {
        c->err.clear();
        return f(c);
    } catch (const std::bad_alloc &) {
        return c->fail(CPTR_ENOMEM, "host allocation failed");
    } catch (...) {
        return c->fail(CPTR_EINVAL, "unexpected host exception");
    }
}

}  // namespace

void model_free(Ctx *c) {
    model_release(static_cast<Model *>(c->model));
    c->model = nullptr;
}

}  // namespace cptr

using namespace cptr;

extern "C" cptr_status cptr_model_set(cptr_ctx *ctx, const cptr_model *model, int32_t on_device) {
    return guard(ctx, [&](Ctx *c) { return model_set(c, model, on_device); });
}

extern "C" cptr_status cptr_assemble(cptr_ctx *ctx, const double *x, const double *xn, double *R, double *J,
                                     double *Se, int32_t on_device) {
    return guard(ctx, [&](Ctx *c) -> cptr_status {
        Model *m = static_cast<Model *>(c->model);
        if (!m) return c->fail(CPTR_ESTATE, "cptr_assemble: no model (cptr_model_set)");
        if (!x || !xn || !R) return c->fail(CPTR_EINVAL, "cptr_assemble: x, xn and R are required");
        const int b = m->dm.b;
        const size_t nb = (size_t)m->n * b, nj = (size_t)m->nnzb * b * b;
        if (on_device) {
            CPTR_TRY(assemble(c, x, xn, R, J, Se));
        } else {
            double *dx = nullptr, *dxn = nullptr, *dR = nullptr, *dJ = nullptr, *dS = nullptr;
            CPTR_TRY(dalloc_t(c, &dx, nb));
            CPTR_TRY(dalloc_t(c, &dxn, nb));
            CPTR_TRY(dalloc_t(c, &dR, nb));
            if (J) CPTR_TRY(dalloc_t(c, &dJ, nj));
            if (Se) CPTR_TRY(dalloc_t(c, &dS, (size_t)m->nnzb));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(dx, x, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
            CPTR_CUDA_TRY(c, cudaMemcpyAsync(dxn, xn, sizeof(double) * nb, cudaMemcpyHostToDevice, c->stream));
            CPTR_TRY(assemble(c, dx, dxn, dR, dJ, dS));
            CPTR_TRY(copy_to_host(c, R, dR, sizeof(double) * nb));
            if (J) CPTR_TRY(copy_to_host(c, J, dJ, sizeof(double) * nj));
            if (Se) CPTR_TRY(copy_to_host(c, Se, dS, sizeof(double) * m->nnzb));
            for (double *p : {dx, dxn, dR, dJ, dS}) dfree(p);
        }
        int32_t e = 0;
        CPTR_TRY(copy_to_host(c, &e, c->flag, sizeof(int32_t)));
        if (e) return c->fail(CPTR_EINVAL, "model assembly: pattern lacks a block");
        CPTR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return CPTR_OK;
    });
}

extern "C" cptr_status cptr_newton(cptr_ctx *ctx, double *x, const double *xn, double rtol_lin, int32_t max_newton,
                                   cptr_newton_stats *st, int32_t on_device) {
    return guard(ctx, [&](Ctx *c) -> cptr_status {
        if (!c->model) return c->fail(CPTR_ESTATE, "cptr_newton: no model (cptr_model_set)");
        if (!x || !xn || max_newton < 1 || !(rtol_lin > 0.0)) return c->fail(CPTR_EINVAL, "cptr_newton: bad arguments");
        return newton(ctx, c, x, xn, rtol_lin, max_newton, st, on_device);
    });
}
