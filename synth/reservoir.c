/*
 * Seeded synthetic input generator: the fully implicit residual, its analytic Jacobian and the
 * discrete Schur-complement operator S_e of a thermal multiphase finite-volume model on a
 * Cartesian grid.  This file produces the *inputs* of the CPTR solver (the linear system and the
 * S_e operator); it holds none of the solver's arithmetic (no decoupling, AMG, ILU or Krylov).
 *
 * Model (Roy, Jonsthovel, Lemon, Wathen, "A constrained pressure-temperature residual (CPTR)
 * method for non-isothermal multiphase flow in porous media", arXiv 1907.04229):
 *   - saturation constraint, the eliminated saturation is S_o            (Sec. 2.1, eq. Sbeta)
 *   - phase mass conservation with Darcy velocity, capillarity ignored   (Sec. 2.1.1, eq. consmass)
 *   - energy advection + conduction, k_T mixing law                      (Sec. 2.1.2, eq. energy3)
 *   - point wells: injector at T_inj, producer at cell T                 (Sec. 2.1.4, eqs. f, fT)
 *   - heaters U (T_heater - T)                                           (Sec. 2.1.4)
 *   - DG(0)/TPFA: harmonic K and k_T, arithmetic face density, phase
 *     upwinding on the sign of the phase potential difference            (Sec. 2.2.1, eqs. conswater,
 *                                                                          consenergy, consoil, upwind)
 *   - implicit Euler                                                     (Sec. 2.2.2, eq. F=0)
 *   - water viscosity (Grabowski) and density (Kell/Trangenstein)        (Appendix A, Tables 3, 4)
 *   - discrete Schur approximation S_e: the energy form with every
 *     coefficient frozen at the current iterate, differentiated only in
 *     the explicit temperature factors                                   (Sec. 3.3.1, eq. Se)
 * Choices the paper leaves open (oil and gas laws, Corey exponent, producer model) are parameters
 * of synth_problem; their values are set by the Python recipes next to this file.
 *
 * Unknowns per cell: u = (p, T, S_w[, S_g]).  Raw equation rows per cell, in this order:
 *   0: water mass, 1: energy, 2: oil mass, 3: gas mass (three-phase only).
 * Jacobian layout: BSR over the 7-point cell graph, columns ascending, b x b blocks row-major,
 * block (r, c) = dR_r / du_c.  Units: kg/s for the mass rows, W for the energy row.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct {
    int32_t nx, ny, nz, nphase;
    double dx, dy, dz;
    double dt, phi, grav;
    const double *kh, *kv;               /* [N] permeability, m^2 (x/y faces use kh, z faces kv) */
    double kT_const;                     /* > 0: constant conductivity; else mixing law */
    double kT_rock, kT_w, kT_o, kT_g;
    double cv_w, cv_o, cv_g, c_rock, rho_rock;
    double mu_o_ref, beta_mu, T0, rho_o_ref, c_o, beta_o, p0;
    double gas_M, mu_g;
    double corey_n;
    int32_t thermal_props_off;           /* 1: rho, mu evaluated at T_props (no T dependence) */
    int32_t n_wells;
    double T_props;
    const int32_t *well_cell, *well_kind;/* kind 0: injector (a = rate m^3/s, c = T_inj);
                                            kind 1: producer (a = WI m^3, c = p_bh Pa) */
    const double *well_a, *well_c;
    const int32_t *heater_cell;
    const double *heater_U, *heater_T;
    int32_t n_heaters, pad_;
} synth_problem;

#define MAXB 4
#define RGAS 8.314462618

typedef struct {
    double S, dS[MAXB];        /* saturation */
    double rho, drho[MAXB];    /* density */
    double lam, dlam[MAXB];    /* mobility k_r / mu */
    double rl, drl[MAXB];      /* rho * lam */
} phase_state;

typedef struct {
    phase_state ph[3];
    double kT, dkT[MAXB];
} cell_state;

static int nunk(const synth_problem *P) { return P->nphase + 1; }
static int raw_row(int phase) { return phase == 0 ? 0 : (phase == 1 ? 2 : 3); }
static double cv_of(const synth_problem *P, int a) { return a == 0 ? P->cv_w : (a == 1 ? P->cv_o : P->cv_g); }

static void water_props(const synth_problem *P, double p, double T, double *rho, double *rp,
                        double *rT, double *mu, double *mT) {
    const double E0 = 999.83952, E1 = 16.955176, E2 = -7.987e-3, E3 = -46.170461e-6,
                 E4 = 105.56302e-9, E5 = -280.54353e-12, E6 = 16.87985e-3, E7 = 10.2,
                 Cw = 3.98854e-4;
    const double A = 2.1850, B = 0.04012, C = 5.1547e-6;
    int off = P->thermal_props_off;
    double Tc = (off ? P->T_props : T) - 273.15;
    double poly = E0 + Tc * (E1 + Tc * (E2 + Tc * (E3 + Tc * (E4 + Tc * E5))));
    double dpoly = E1 + Tc * (2 * E2 + Tc * (3 * E3 + Tc * (4 * E4 + Tc * 5 * E5)));
    double den = 1.0 + E6 * Tc;
    double f = poly / den, df = (dpoly * den - poly * E6) / (den * den);
    double ex = exp(Cw * (p * 1e-6 - E7));
    *rho = f * ex;
    *rp = *rho * Cw * 1e-6;
    *rT = off ? 0.0 : df * ex;
    double TF = Tc * 1.8 + 32.0;
    double q = -1.0 + B * TF + C * TF * TF;
    *mu = 1e-3 * A / q;
    *mT = off ? 0.0 : -1e-3 * A * (B + 2.0 * C * TF) * 1.8 / (q * q);
}

static void cell_eval(const synth_problem *P, const double *u, cell_state *cs) {
    int b = nunk(P);
    double p = u[0], T = u[1];
    double Sw = u[2], Sg = (P->nphase == 3) ? u[3] : 0.0;
    memset(cs, 0, sizeof(*cs));
    for (int a = 0; a < P->nphase; ++a) {
        phase_state *s = &cs->ph[a];
        double rho, rp, rT, mu, mT;
        if (a == 0) {
            water_props(P, p, T, &rho, &rp, &rT, &mu, &mT);
            s->S = Sw; s->dS[2] = 1.0;
        } else if (a == 1) {
            double Te = P->thermal_props_off ? P->T_props : T;
            rho = P->rho_o_ref * exp(P->c_o * (p - P->p0) - P->beta_o * (Te - P->T0));
            rp = P->c_o * rho;
            rT = P->thermal_props_off ? 0.0 : -P->beta_o * rho;
            mu = P->mu_o_ref * exp(-P->beta_mu * (Te - P->T0));
            mT = P->thermal_props_off ? 0.0 : -P->beta_mu * mu;
            s->S = 1.0 - Sw - Sg; s->dS[2] = -1.0; if (b == 4) s->dS[3] = -1.0;
        } else {
            double Te = P->thermal_props_off ? P->T_props : T;
            rho = p * P->gas_M / (RGAS * Te);
            rp = P->gas_M / (RGAS * Te);
            rT = P->thermal_props_off ? 0.0 : -rho / Te;
            mu = P->mu_g; mT = 0.0;
            s->S = Sg; s->dS[3] = 1.0;
        }
        s->rho = rho; s->drho[0] = rp; s->drho[1] = rT;
        /* Corey relative permeability k_r = max(S,0)^n */
        double Sc = s->S > 0.0 ? s->S : 0.0;
        double kr = pow(Sc, P->corey_n);
        double dkr = (s->S > 0.0) ? P->corey_n * pow(Sc, P->corey_n - 1.0) : 0.0;
        s->lam = kr / mu;
        for (int c = 0; c < b; ++c) s->dlam[c] = dkr * s->dS[c] / mu;
        s->dlam[1] += -kr * mT / (mu * mu);
        s->rl = rho * s->lam;
        for (int c = 0; c < b; ++c) s->drl[c] = s->drho[c] * s->lam + rho * s->dlam[c];
    }
    if (P->kT_const > 0.0) {
        cs->kT = P->kT_const;
    } else {
        double kf[3] = {P->kT_w, P->kT_o, P->kT_g};
        cs->kT = (1.0 - P->phi) * P->kT_rock;
        for (int a = 0; a < P->nphase; ++a) {
            cs->kT += P->phi * cs->ph[a].S * kf[a];
            for (int c = 0; c < b; ++c) cs->dkT[c] += P->phi * kf[a] * cs->ph[a].dS[c];
        }
    }
}

/* Number of block nonzeros of the 7-point cell graph (diagonal included). */
int64_t synth_nnzb(const synth_problem *P) {
    int64_t nx = P->nx, ny = P->ny, nz = P->nz;
    int64_t faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
    return nx * ny * nz + 2 * faces;
}

/* Cell-graph pattern, rows in natural order i = x + nx (y + ny z), columns ascending. */
void synth_pattern(const synth_problem *P, int32_t *row_ptr, int32_t *col_idx) {
    int32_t nx = P->nx, ny = P->ny, nz = P->nz, nxy = nx * ny;
    int64_t k = 0;
    row_ptr[0] = 0;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x) {
                int32_t i = x + nx * (y + ny * z);
                if (z > 0) col_idx[k++] = i - nxy;
                if (y > 0) col_idx[k++] = i - nx;
                if (x > 0) col_idx[k++] = i - 1;
                col_idx[k++] = i;
                if (x < nx - 1) col_idx[k++] = i + 1;
                if (y < ny - 1) col_idx[k++] = i + nx;
                if (z < nz - 1) col_idx[k++] = i + nxy;
                row_ptr[i + 1] = (int32_t)k;
            }
}

static int64_t find_blk(const int32_t *rp, const int32_t *ci, int32_t i, int32_t j) {
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (ci[k] == j) return k;
    return -1;
}

static double harm(double a, double b) { return 2.0 * a * b / (a + b); }

/*
 * Residual R (raw rows, [N*b]) of the implicit Euler step from state xn to state x.
 * If J != NULL, the analytic Jacobian dR/dx is written into J ([nnzb*b*b], pattern from
 * synth_pattern).  If Se != NULL, the S_e operator ([nnzb] scalars on the same pattern) is
 * written.  Returns 0, or -1 on an inconsistent pattern.
 */
int synth_assemble(const synth_problem *P, const double *x, const double *xn,
                   const int32_t *rp, const int32_t *ci, double *R, double *J, double *Se) {
    const int b = nunk(P), bb = b * b, np = P->nphase;
    const int32_t nx = P->nx, ny = P->ny, nz = P->nz, nxy = nx * ny;
    const int64_t N = (int64_t)nx * ny * nz;
    const double V = P->dx * P->dy * P->dz;
    memset(R, 0, sizeof(double) * N * b);
    if (J) memset(J, 0, sizeof(double) * rp[N] * bb);
    if (Se) memset(Se, 0, sizeof(double) * rp[N]);

    /* accumulation, wells, heaters: cell terms */
    for (int64_t i = 0; i < N; ++i) {
        cell_state cs, cn;
        const double *u = x + i * b, *un = xn + i * b;
        cell_eval(P, u, &cs);
        cell_eval(P, un, &cn);
        int64_t kd = find_blk(rp, ci, (int32_t)i, (int32_t)i);
        if (kd < 0) return -1;
        double *Jd = J ? J + kd * bb : NULL;
        double *Ri = R + i * b;
        const double T = u[1], Tn = un[1];
        double acc = V / P->dt;
        /* phase mass: V phi (rho S - rho^n S^n) / dt */
        double eacc = 0.0;
        for (int a = 0; a < np; ++a) {
            const phase_state *s = &cs.ph[a], *sn = &cn.ph[a];
            double cv = cv_of(P, a);
            Ri[raw_row(a)] += acc * P->phi * (s->rho * s->S - sn->rho * sn->S);
            eacc += P->phi * cv * (s->rho * s->S * T - sn->rho * sn->S * Tn);
            if (Jd)
                for (int c = 0; c < b; ++c) {
                    double dm = s->drho[c] * s->S + s->rho * s->dS[c];
                    Jd[raw_row(a) * b + c] += acc * P->phi * dm;
                    Jd[1 * b + c] += acc * P->phi * cv * (dm * T + (c == 1 ? s->rho * s->S : 0.0));
                }
            if (Se) Se[kd] += acc * P->phi * cv * s->S * s->rho;
        }
        eacc += (1.0 - P->phi) * P->rho_rock * P->c_rock * (T - Tn);
        Ri[1] += acc * eacc;
        if (Jd) Jd[1 * b + 1] += acc * (1.0 - P->phi) * P->rho_rock * P->c_rock;
        if (Se) Se[kd] += acc * (1.0 - P->phi) * P->rho_rock * P->c_rock;
    }
    for (int w = 0; w < P->n_wells; ++w) {
        int32_t i = P->well_cell[w];
        int64_t kd = find_blk(rp, ci, i, i);
        const double *u = x + (int64_t)i * b;
        double *Ri = R + (int64_t)i * b;
        double *Jd = J ? J + kd * bb : NULL;
        if (P->well_kind[w] == 0) {
            /* injector: water at T_inj, mass source q rho_w(p, T_inj) */
            double q = P->well_a[w], Tinj = P->well_c[w];
            double rho, rp_, rT, mu, mT;
            water_props(P, u[0], Tinj, &rho, &rp_, &rT, &mu, &mT);
            Ri[0] -= q * rho;
            Ri[1] -= P->cv_w * Tinj * q * rho;
            if (Jd) {
                Jd[0 * b + 0] -= q * rp_;
                Jd[1 * b + 0] -= P->cv_w * Tinj * q * rp_;
            }
        } else {
            /* producer: q_alpha = WI lam_alpha (p - p_bh)^+, mass sink rho_alpha q_alpha */
            double WI = P->well_a[w], pbh = P->well_c[w];
            double dp = u[0] - pbh;
            if (dp <= 0.0) continue;
            cell_state cs;
            cell_eval(P, u, &cs);
            double T = u[1];
            for (int a = 0; a < np; ++a) {
                const phase_state *s = &cs.ph[a];
                double cv = cv_of(P, a);
                double m = WI * s->rl * dp;
                Ri[raw_row(a)] += m;
                Ri[1] += cv * T * m;
                if (Jd)
                    for (int c = 0; c < b; ++c) {
                        double dm = WI * dp * s->drl[c] + (c == 0 ? WI * s->rl : 0.0);
                        Jd[raw_row(a) * b + c] += dm;
                        Jd[1 * b + c] += cv * (T * dm + (c == 1 ? m : 0.0));
                    }
                if (Se) Se[kd] += cv * m;
            }
        }
    }
    for (int h = 0; h < P->n_heaters; ++h) {
        int32_t i = P->heater_cell[h];
        int64_t kd = find_blk(rp, ci, i, i);
        double U = P->heater_U[h];
        R[(int64_t)i * b + 1] -= U * (P->heater_T[h] - x[(int64_t)i * b + 1]);
        if (J) J[kd * bb + 1 * b + 1] += U;
        if (Se) Se[kd] += U;
    }

    /* facet terms: each interior face once, L = lower index, R = upper index */
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t xx = 0; xx < nx; ++xx) {
                int32_t L = xx + nx * (y + ny * z);
                for (int dir = 0; dir < 3; ++dir) {
                    int32_t Rc;
                    double area, dist, dzLR, KL, KR;
                    if (dir == 0) {
                        if (xx == nx - 1) continue;
                        Rc = L + 1; area = P->dy * P->dz; dist = P->dx; dzLR = 0.0;
                        KL = P->kh[L]; KR = P->kh[Rc];
                    } else if (dir == 1) {
                        if (y == ny - 1) continue;
                        Rc = L + nx; area = P->dx * P->dz; dist = P->dy; dzLR = 0.0;
                        KL = P->kh[L]; KR = P->kh[Rc];
                    } else {
                        if (z == nz - 1) continue;
                        Rc = L + nxy; area = P->dx * P->dy; dist = P->dz;
                        dzLR = -P->dz; /* depth grows with z: z_L - z_R = -dz */
                        KL = P->kv[L]; KR = P->kv[Rc];
                    }
                    const double *uL = x + (int64_t)L * b, *uR = x + (int64_t)Rc * b;
                    cell_state sL, sR;
                    cell_eval(P, uL, &sL);
                    cell_eval(P, uR, &sR);
                    double Ups = area / dist * harm(KL, KR);
                    int64_t kLL = find_blk(rp, ci, L, L), kLR = find_blk(rp, ci, L, Rc);
                    int64_t kRL = find_blk(rp, ci, Rc, L), kRR = find_blk(rp, ci, Rc, Rc);
                    if (kLR < 0 || kRL < 0) return -1;
                    double *RL = R + (int64_t)L * b, *RR = R + (int64_t)Rc * b;
                    for (int a = 0; a < np; ++a) {
                        const phase_state *pL = &sL.ph[a], *pR = &sR.ph[a];
                        double cv = cv_of(P, a);
                        double rbar = 0.5 * (pL->rho + pR->rho);
                        double Phi = (uL[0] - uR[0]) - rbar * P->grav * dzLR;
                        int upL = Phi >= 0.0; /* tie: lower-index cell */
                        const phase_state *pu = upL ? pL : pR;
                        double Tup = upL ? uL[1] : uR[1];
                        double F = Ups * pu->rl * Phi;
                        int ra = raw_row(a);
                        RL[ra] += F; RR[ra] -= F;
                        RL[1] += cv * Tup * F; RR[1] -= cv * Tup * F;
                        if (J) {
                            double dFL[MAXB], dFR[MAXB];
                            for (int c = 0; c < b; ++c) {
                                double dPhiL = (c == 0 ? 1.0 : 0.0) - 0.5 * pL->drho[c] * P->grav * dzLR;
                                double dPhiR = (c == 0 ? -1.0 : 0.0) - 0.5 * pR->drho[c] * P->grav * dzLR;
                                dFL[c] = Ups * (pu->rl * dPhiL + (upL ? Phi * pL->drl[c] : 0.0));
                                dFR[c] = Ups * (pu->rl * dPhiR + (upL ? 0.0 : Phi * pR->drl[c]));
                            }
                            for (int c = 0; c < b; ++c) {
                                double dGL = cv * (Tup * dFL[c] + ((upL && c == 1) ? F : 0.0));
                                double dGR = cv * (Tup * dFR[c] + ((!upL && c == 1) ? F : 0.0));
                                J[kLL * bb + ra * b + c] += dFL[c];
                                J[kLR * bb + ra * b + c] += dFR[c];
                                J[kRL * bb + ra * b + c] -= dFL[c];
                                J[kRR * bb + ra * b + c] -= dFR[c];
                                J[kLL * bb + 1 * b + c] += dGL;
                                J[kLR * bb + 1 * b + c] += dGR;
                                J[kRL * bb + 1 * b + c] -= dGL;
                                J[kRR * bb + 1 * b + c] -= dGR;
                            }
                        }
                        if (Se) {
                            /* frozen mass flux F advects delta T from the upwind cell */
                            int64_t kLu = upL ? kLL : kLR, kRu = upL ? kRL : kRR;
                            Se[kLu] += cv * F;
                            Se[kRu] -= cv * F;
                        }
                    }
                    /* conduction: harmonic k_T */
                    double kh_T = harm(sL.kT, sR.kT);
                    double UT = area / dist * kh_T;
                    double dT = uL[1] - uR[1];
                    RL[1] += UT * dT; RR[1] -= UT * dT;
                    if (J) {
                        double s2 = (sL.kT + sR.kT) * (sL.kT + sR.kT);
                        double dhL = 2.0 * sR.kT * sR.kT / s2, dhR = 2.0 * sL.kT * sL.kT / s2;
                        for (int c = 0; c < b; ++c) {
                            double gL = area / dist * dhL * sL.dkT[c] * dT + (c == 1 ? UT : 0.0);
                            double gR = area / dist * dhR * sR.dkT[c] * dT - (c == 1 ? UT : 0.0);
                            J[kLL * bb + 1 * b + c] += gL;
                            J[kLR * bb + 1 * b + c] += gR;
                            J[kRL * bb + 1 * b + c] -= gL;
                            J[kRR * bb + 1 * b + c] -= gR;
                        }
                    }
                    if (Se) {
                        Se[kLL] += UT; Se[kLR] -= UT;
                        Se[kRR] += UT; Se[kRL] -= UT;
                    }
                }
            }
    return 0;
}

/* Evaluate water density/viscosity (the printed correlations) for tests: out = {rho, mu}. */
void synth_water(double p, double T, double *out) {
    synth_problem P;
    memset(&P, 0, sizeof(P));
    double rp, rT, mT;
    water_props(&P, p, T, &out[0], &rp, &rT, &out[1], &mT);
}
