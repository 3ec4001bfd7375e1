/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the coupled lattice-Boltzmann
 * time step and the wall-link boundary schemes of Li, Chan, Feng & Wang,
 * "Lattice Boltzmann Boundary Conditions for Flow, Convection-Diffusion and MHD
 * Simulations" (arXiv 2506.00907).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * Form: push ("relax, then propagate") exactly as written in Eq. 1, 3 and 5:
 *   1. moments at t of every fluid node              (Eq. 2, 4, 6 and Sec. 2)
 *   2. equilibria and relaxation                     (Eq. 1-6)
 *   3. propagation to x + e_a for fluid targets      (Eq. 1, 3, 5)
 *   4. every wall link writes the unknown population at its node A
 *      (Sec. 3-4, Eq. 11-29, 34-35, 43), each link independently (pair-wise);
 *      two comparison schemes of the paper are selectable per link: Eq. 15/16
 *      for every d (Sec. 5.1) and the simplified flux wall of Eq. 33 (Sec. 5.4);
 *      open boundaries (Sec. 5.1): given velocity is the velocity kind with a
 *      normal u (Eq. 41, 43), given pressure its own kind (Eq. 42, 44);
 *      a reaction flux of C nonlinear in C_X (rational form) by the M scheme;
 *      several concentration species (Sec. 4.2.2, text after Eq. 23): each
 *      species' C_i(X) by Eq. 13, the surface reaction fluxes F_i(C_1, C_2, ..)
 *      of a mass-action network evaluated explicitly from them, and each F_i
 *      added to its own species by the M scheme (Eq. 23-27), with no coupled
 *      (Newton) solve.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes of the repository):
 *   - D2Q5 / D3Q7 weights: w0 = 1/2, 1/8 (2D); w0 = 1/4, 1/8 (3D); c_h^2 = c_g^2 = 1/4.
 *     The paper's parameter sets (Sec. 5.3, 5.4, 6) all give c_h^2/c^2 = 1/4.
 *   - body force: Guo-Zheng-Shi forcing (Sec. 2.4 says only that the right-hand
 *     side of Eq. 1 "can be modified").
 *   - Lorentz force: magnetic (Maxwell) stress 1/2|B|^2 I - BB added to the second
 *     moment of f^eq, mu = 1 (Sec. 2.3 says only "some modifications").
 *   - E solid (no second fluid node): the link is evaluated at d = 0.5 with
 *     phi(E) := phi(A), which needs no E.
 *   - the fluid velocity entering boundary equilibria is the wall velocity u_w
 *     stored in the link (walls are never extrapolated for u).
 *   - simplified flux wall for d != 1 (Eq. 33 is printed for d = 1 only): the
 *     increments join the bounced population in the interpolation of Eq. 11/12,
 *     which is Eq. 33 at d = 1 and Eq. 28 at d = 1/2.
 *   - given pressure for d < 1/2 (Eq. 42/44 are printed for d = 1/2 and d >= 1/2):
 *     the interpolation of Eq. 16 to Y, as for a given C (Eq. 19/20); u(X) is
 *     extrapolated by Eq. 13; the pressure kind belongs to flow-only cases (the
 *     paper's open channel), not to cases with a concentration or a magnetic field.
 * Lattice units throughout: dx = dt = 1, c = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Lattices (Sec. 2.1: D2Q9 / D3Q19 [Qian 1992]; Sec. 2.2-2.3: D2Q5 / D3Q7).  */
/* Direction numbering (an interface shared with the C-ABI by specification): */
/* D2Q9: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-)   */
/* D2Q5: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y                                       */
/* D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z, 7 (+x+y), 8 (-x-y),     */
/*   9 (+x-y), 10 (-x+y), 11 (+x+z), 12 (-x-z), 13 (+x-z), 14 (-x+z),         */
/*   15 (+y+z), 16 (-y-z), 17 (+y-z), 18 (-y+z)                               */
/* D3Q7: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z                           */
/* ------------------------------------------------------------------------- */
static const int D2Q9_E[9][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0},
                                 {1,1,0},{-1,1,0},{-1,-1,0},{1,-1,0}};
static const double D2Q9_W[9] = {4.0/9, 1.0/9, 1.0/9, 1.0/9, 1.0/9,
                                 1.0/36, 1.0/36, 1.0/36, 1.0/36};
static const int D2Q5_E[5][3] = {{0,0,0},{1,0,0},{0,1,0},{-1,0,0},{0,-1,0}};
static const double D2Q5_W[5] = {0.5, 0.125, 0.125, 0.125, 0.125};
static const int D3Q19_E[19][3] = {{0,0,0},
    {1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1},
    {1,1,0},{-1,-1,0},{1,-1,0},{-1,1,0},
    {1,0,1},{-1,0,-1},{1,0,-1},{-1,0,1},
    {0,1,1},{0,-1,-1},{0,1,-1},{0,-1,1}};
static const double D3Q19_W[19] = {1.0/3,
    1.0/18, 1.0/18, 1.0/18, 1.0/18, 1.0/18, 1.0/18,
    1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36,
    1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36, 1.0/36};
static const int D3Q7_E[7][3] = {{0,0,0},{1,0,0},{-1,0,0},{0,1,0},{0,-1,0},{0,0,1},{0,0,-1}};
static const double D3Q7_W[7] = {0.25, 0.125, 0.125, 0.125, 0.125, 0.125, 0.125};

static const double CS2 = 1.0 / 3.0;   /* c_s^2 for D2Q9 / D3Q19 */
static const double CH2 = 0.25;        /* c_h^2 = c_g^2 for D2Q5 / D3Q7 */

typedef struct {
    int q;
    const int (*e)[3];
    const double *w;
} lattice;

static lattice flow_lattice(int dim) {
    lattice L;
    if (dim == 2) { L.q = 9; L.e = D2Q9_E; L.w = D2Q9_W; }
    else          { L.q = 19; L.e = D3Q19_E; L.w = D3Q19_W; }
    return L;
}
static lattice scalar_lattice(int dim) {
    lattice L;
    if (dim == 2) { L.q = 5; L.e = D2Q5_E; L.w = D2Q5_W; }
    else          { L.q = 7; L.e = D3Q7_E; L.w = D3Q7_W; }
    return L;
}
/* the opposite direction a' with e_a' = -e_a, found by search */
static int opposite(lattice L, int a) {
    for (int b = 0; b < L.q; ++b)
        if (L.e[b][0] == -L.e[a][0] && L.e[b][1] == -L.e[a][1] && L.e[b][2] == -L.e[a][2])
            return b;
    return -1;
}
static double edot(lattice L, int a, const double v[3]) {
    return L.e[a][0] * v[0] + L.e[a][1] * v[1] + L.e[a][2] * v[2];
}

/* ------------------------------------------------------------------------- */
/* Equilibria                                                                 */
/* ------------------------------------------------------------------------- */
/* Eq. 2 (flow), plus the magnetic stress of the Lorentz-force reading:
 *   f^eq_a = rho w_a [1 + e.u/cs2 + (e.u)^2/(2 cs2^2) - u.u/(2 cs2)]
 *          + w_a [ (1/2|B|^2 I - BB) : (e e - cs2 I) ] / (2 cs2^2)
 * dim = 2 or 3 (trace of I).  B may be NULL (no magnetic field). */
double orc_feq(int dim, int a, double rho, const double u[3], const double B[3]) {
    lattice L = flow_lattice(dim);
    double eu = edot(L, a, u);
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double feq = rho * L.w[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    if (B) {
        double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        double eB = edot(L, a, B);
        double ee = (double)(L.e[a][0] * L.e[a][0] + L.e[a][1] * L.e[a][1] + L.e[a][2] * L.e[a][2]);
        /* (1/2|B|^2 I) : (ee - cs2 I) = 1/2|B|^2 (|e|^2 - dim cs2) */
        double iso = 0.5 * BB * (ee - dim * CS2);
        /* (BB) : (ee - cs2 I) = (e.B)^2 - cs2 |B|^2 */
        double bb = eB * eB - CS2 * BB;
        feq += L.w[a] * (iso - bb) / (2.0 * CS2 * CS2);
    }
    return feq;
}

/* Eq. 4: h^eq_a = C w_a [1 + e.u / c_h^2] */
double orc_heq(int dim, int a, double C, const double u[3]) {
    lattice L = scalar_lattice(dim);
    return C * L.w[a] * (1.0 + edot(L, a, u) / CH2);
}

/* Eq. 6, component k: g^eq_{a,k} = w_a [B_k + ((e.u) B_k - (e.B) u_k) / c_g^2] */
double orc_geq(int dim, int a, int k, const double B[3], const double u[3]) {
    lattice L = scalar_lattice(dim);
    return L.w[a] * (B[k] + (edot(L, a, u) * B[k] - edot(L, a, B) * u[k]) / CH2);
}

/* Guo forcing source (body-force reading), already weighted by (1 - 1/(2 tau)):
 *   S_a = (1 - 1/(2 tau)) w_a [ (e_a - u)/cs2 + (e_a.u) e_a / cs2^2 ] . F */
double orc_guo(int dim, int a, double tau, const double u[3], const double F[3]) {
    lattice L = flow_lattice(dim);
    double eu = edot(L, a, u);
    double s = 0.0;
    for (int k = 0; k < 3; ++k)
        s += ((L.e[a][k] - u[k]) / CS2 + eu * L.e[a][k] / (CS2 * CS2)) * F[k];
    return (1.0 - 1.0 / (2.0 * tau)) * L.w[a] * s;
}

/* lattice tables for tests */
int orc_lattice(int dim, int scalar, int *q, int *e /* q*3 */, double *w) {
    lattice L = scalar ? scalar_lattice(dim) : flow_lattice(dim);
    *q = L.q;
    for (int a = 0; a < L.q; ++a) {
        for (int k = 0; k < 3; ++k) e[3 * a + k] = L.e[a][k];
        w[a] = L.w[a];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Wall links                                                                 */
/* ------------------------------------------------------------------------- */
enum { ORC_F = 0, ORC_H = 1, ORC_G0 = 2,               /* field: f, h (species 0), g_k = 2 + k */
       ORC_HS1 = 5 };                                   /* species k >= 1 of C: field 4 + k (5, 6, 7) */
#define ORC_MAX_SPECIES 4
#define ORC_MAX_REACT 4
/* species index of a concentration field, or -1 */
static int species_of(int field) {
    if (field == ORC_H) return 0;
    if (field >= ORC_HS1 && field < ORC_HS1 + ORC_MAX_SPECIES - 1) return field - ORC_HS1 + 1;
    return -1;
}
enum { ORC_VELOCITY = 0, ORC_GIVEN = 1, ORC_FLUX = 2, ORC_NEUMANN_BFL = 3,
       ORC_VELOCITY_EQ15 = 4,   /* Eq. 15 with Eq. 16 for every d (the paper's own scheme before Eq. 43) */
       ORC_FLUX_SIMPLIFIED = 5, /* flux and move increments added to the bounced population at X (Eq. 33) */
       ORC_PRESSURE = 6,        /* given density (pressure) of an open boundary, Eq. 42 and 44 */
       ORC_FLUX_RATIONAL = 7,   /* M scheme with the nonlinear flux (k0 + k1 phi_X) / (1 + phi_wall phi_X) */
       ORC_REACTION = 8         /* M scheme with k0 + k1 R_i(C_X) of the surface reaction network */ };

/* Mass-action surface reactions: reaction j runs at rate_j prod_m C_m^order[j][m]
 * per unit wall area and time; species i is produced at
 * R_i = sum_j stoich[j][i] rate_j prod_m C_m^order[j][m]. */
typedef struct {
    int n;
    double rate[ORC_MAX_REACT];
    int order[ORC_MAX_REACT][ORC_MAX_SPECIES];
    double stoich[ORC_MAX_REACT][ORC_MAX_SPECIES];
} orc_network;

/* R_i at the concentrations C[0 .. nspecies-1] */
static double network_rate(const orc_network *net, int nspecies, int i, const double *C) {
    double R = 0.0;
    for (int j = 0; j < net->n; ++j) {
        double r = net->rate[j];
        for (int m = 0; m < nspecies; ++m)
            for (int o = 0; o < net->order[j][m]; ++o) r *= C[m];
        R += net->stoich[j][i] * r;
    }
    return R;
}

typedef struct {
    int32_t node;        /* first fluid node A */
    int32_t field;       /* ORC_F, ORC_H, ORC_G0 + k */
    int32_t dir;         /* unknown direction a at A (pointing from the wall into the fluid) */
    int32_t kind;        /* ORC_VELOCITY ... */
    double d;            /* AX / |EA| in (0, 1] (Eq. 13) */
    double u_wall[3];    /* wall velocity */
    double phi_wall;     /* given C or B_k (GIVEN) */
    double k0, k1;       /* flux increment per step: dphi_flux = k0 + k1 * phi_X (Eq. 23, 48) */
} orc_link;

/* Everything a link formula reads, at time t.  For the flow field phi is rho. */
typedef struct {
    double p_a_A;        /* p_rel,a(A,t)   (unknown direction, at A)  */
    double p_ap_A;       /* p_rel,a'(A,t)  (toward the wall, at A)     */
    double p_ap_E;       /* p_rel,a'(E,t)                              */
    double phi_A, phi_E; /* rho (f), C (h) or B_k (g_k) at A and E     */
    double B_A[3], B_E[3]; /* full B at A and E (g fields only)        */
    double u_A[3], u_E[3]; /* fluid velocity at A and E (f field only)  */
    double C_A[ORC_MAX_SPECIES], C_E[ORC_MAX_SPECIES]; /* every species' C at A and E (reaction links) */
    int nspecies;
    const orc_network *net;
} orc_link_in;

/* Eq. 13: extrapolation of an unknown macroscopic quantity to the wall point X */
static double extrap_X(double d, double phiE, double phiA) {
    return (-d) * phiE + (d + 1.0) * phiA;
}

/* Interpolation / extrapolation to the mirror point Y (Eq. 16, 20, 35) */
static double at_Y(double d, double pE, double pA) {
    return (1.0 - 2.0 * d) * pE + (2.0 * d) * pA;
}

/* The new unknown population p_a(A, t+1) for one link (dim 2/3). */
double orc_eval_link(int dim, const orc_link *lk, const orc_link_in *in) {
    double d = lk->d;
    if (lk->field == ORC_F) {
        lattice L = flow_lattice(dim);
        int a = lk->dir, ap = opposite(L, a);
        /* rho(X,t) by Eq. 13; u(X) = wall velocity.  Increment f^eq_a(X) - f^eq_a'(X)
         * with Eq. 2 (magnetic terms are even in e and cancel). */
        double rhoX = extrap_X(d, in->phi_E, in->phi_A);
        double incr = orc_feq(dim, a, rhoX, lk->u_wall, NULL) - orc_feq(dim, ap, rhoX, lk->u_wall, NULL);
        if (lk->kind == ORC_PRESSURE) {
            /* Given density rho_w = phi_wall (pressure rho_w c_s^2) on an open
             * boundary.  Zeroth-moment pair conservation (the flow form of
             * Eq. 18-19): p_a(A) = f^eq_a(X) + f^eq_a'(X) - f_rel,a'(Y), with
             * u(X,t) extrapolated by Eq. 13 (the outlet velocity is unknown) and
             * Y by Eq. 16 for d < 1/2; Eq. 44 for d >= 1/2; both are Eq. 42 at
             * d = 1/2. */
            double uX[3];
            for (int c = 0; c < 3; ++c) uX[c] = extrap_X(d, in->u_E[c], in->u_A[c]);
            double sum_eq = orc_feq(dim, a, lk->phi_wall, uX, NULL) + orc_feq(dim, ap, lk->phi_wall, uX, NULL);
            if (d < 0.5) return sum_eq - at_Y(d, in->p_ap_E, in->p_ap_A);
            return ((2.0 * d - 1.0) * in->p_a_A - in->p_ap_A + sum_eq) / (2.0 * d);
        }
        if (lk->kind == ORC_VELOCITY_EQ15) {
            /* Eq. 15 with Eq. 16 for every d in (0, 1]: extrapolation to Y for
             * d >= 0.5, which Sec. 5.1 reports unstable for d above about 0.8 */
            return incr + at_Y(d, in->p_ap_E, in->p_ap_A);
        }
        if (lk->kind != ORC_VELOCITY) return NAN;
        if (d < 0.5) {
            /* Eq. 15 with Eq. 16 */
            return incr + at_Y(d, in->p_ap_E, in->p_ap_A);
        }
        /* Eq. 43 (d >= 0.5); with u_wall = 0 this is Eq. 12 */
        return ((2.0 * d - 1.0) * in->p_a_A + in->p_ap_A + incr) / (2.0 * d);
    }
    lattice L = scalar_lattice(dim);
    int a = lk->dir, ap = opposite(L, a);
    int is_g = species_of(lk->field) < 0;
    int k = is_g ? lk->field - ORC_G0 : 0;
    const double *uw = lk->u_wall;
    switch (lk->kind) {
    case ORC_GIVEN: {
        /* Eq. 19 (h) / Eq. 34 (g_k) with Y from Eq. 20 / 35 */
        double pY = at_Y(d, in->p_ap_E, in->p_ap_A);
        if (!is_g) {
            double C = lk->phi_wall;
            return orc_heq(dim, a, C, uw) + orc_heq(dim, ap, C, uw) - pY;
        }
        double BX[3];
        for (int c = 0; c < 3; ++c) BX[c] = extrap_X(d, in->B_E[c], in->B_A[c]);
        BX[k] = lk->phi_wall;
        return orc_geq(dim, a, k, BX, uw) + orc_geq(dim, ap, k, BX, uw) - pY;
    }
    case ORC_FLUX:
    case ORC_FLUX_RATIONAL:
    case ORC_REACTION: {
        /* M scheme, Eq. 25-27, with the flux increment (Eq. 23) and the
         * moving-wall correction (Eq. 24) evaluated at X (Eq. 13).  A reaction
         * flux nonlinear in C is evaluated explicitly at C_X (Sec. 4.2.2): the
         * rational form (k0 + k1 C_X) / (1 + K C_X), K = phi_wall, or the
         * network's R_i of every species' C_X (each by Eq. 13 from its own C at
         * A and E). */
        double phiX = extrap_X(d, in->phi_E, in->phi_A);
        double dflux;
        if (lk->kind == ORC_FLUX_RATIONAL) {
            dflux = (lk->k0 + lk->k1 * phiX) / (1.0 + lk->phi_wall * phiX);
        } else if (lk->kind == ORC_REACTION) {
            double CX[ORC_MAX_SPECIES];
            for (int m = 0; m < in->nspecies; ++m) CX[m] = extrap_X(d, in->C_E[m], in->C_A[m]);
            if (!in->net || is_g) return NAN;
            dflux = lk->k0 + lk->k1 * network_rate(in->net, in->nspecies, species_of(lk->field), CX);
        } else {
            dflux = lk->k0 + lk->k1 * phiX;
        }
        double minus_u[3] = {-uw[0], -uw[1], -uw[2]};
        double dmove;
        if (!is_g) {
            dmove = orc_heq(dim, ap, phiX, minus_u) - orc_heq(dim, a, phiX, minus_u);
        } else {
            double BX[3];
            for (int c = 0; c < 3; ++c) BX[c] = extrap_X(d, in->B_E[c], in->B_A[c]);
            dmove = orc_geq(dim, ap, k, BX, minus_u) - orc_geq(dim, a, k, BX, minus_u);
        }
        double pM_rel = (0.5 - d) * in->p_ap_E + (0.5 + d) * in->p_ap_A;   /* Eq. 25 */
        double pM_new = pM_rel + dflux + dmove;                              /* Eq. 26 */
        double pE_new = in->p_a_A;                 /* p_a(E,t+1) = p_rel,a(A,t) */
        return ((d - 0.5) * pE_new + pM_new) / (d + 0.5);                    /* Eq. 27 */
    }
    case ORC_FLUX_SIMPLIFIED: {
        /* Eq. 33: the flux increment (Eq. 23) and the moving-wall correction
         * (Eq. 24), both at phi_X of Eq. 13, are added to the population bounced
         * at the wall point X, and A is reached by the interpolation of Eq. 11/12
         * (Eq. 21/22 without flux).  At d = 1 this is Eq. 33 as printed; at d = 1/2
         * it is Eq. 28. */
        double phiX = extrap_X(d, in->phi_E, in->phi_A);
        double dflux = lk->k0 + lk->k1 * phiX;
        double minus_u[3] = {-uw[0], -uw[1], -uw[2]};
        double dmove;
        if (!is_g) {
            dmove = orc_heq(dim, ap, phiX, minus_u) - orc_heq(dim, a, phiX, minus_u);
        } else {
            double BX[3];
            for (int c = 0; c < 3; ++c) BX[c] = extrap_X(d, in->B_E[c], in->B_A[c]);
            dmove = orc_geq(dim, ap, k, BX, minus_u) - orc_geq(dim, a, k, BX, minus_u);
        }
        if (d < 0.5) return at_Y(d, in->p_ap_E, in->p_ap_A) + dflux + dmove;
        return ((2.0 * d - 1.0) * in->p_a_A + in->p_ap_A + dflux + dmove) / (2.0 * d);
    }
    case ORC_NEUMANN_BFL:
        if (d < 0.5) return at_Y(d, in->p_ap_E, in->p_ap_A);                 /* Eq. 21 */
        return ((2.0 * d - 1.0) * in->p_a_A + in->p_ap_A) / (2.0 * d);      /* Eq. 22 */
    default:
        return NAN;
    }
}

/* ------------------------------------------------------------------------- */
/* Simulation state                                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int dim, nx, ny, nz, has_h, has_g, nB;
    int nC;                    /* concentration species (0, or 1..ORC_MAX_SPECIES with has_h) */
    long N;
    double tau_nu, tau_D, tau_eta;
    double tau_Ds[ORC_MAX_SPECIES]; /* tau_D of each species (species 0: tau_D) */
    double C0s[ORC_MAX_SPECIES];    /* initial C of species 1.. (species 0: orc_init's C0) */
    orc_network net;           /* surface reactions of ORC_REACTION links */
    double accel[3];           /* body force per unit mass: F = rho * accel */
    uint8_t *solid;
    double *f, *h, *g;         /* populations at t (after propagation, before relaxation); h: [nC][qm][N] */
    double *fr, *hr, *gr;      /* relaxed populations at t */
    double *fn, *hn, *gn;      /* populations at t+1 */
    double *rho, *u, *C, *B;   /* moments at t: rho[N], u[3N], C[nC][N], B[3N] */
    int32_t *nbf, *nbm;        /* neighbour tables: node of x + e_a, [a * N + n] */
    orc_link *links;
    long nlinks;
    long steps;
    int motion;                /* wall motion (Sec. 5.2): velocity links of f move with u_wall cos(omega t + phase) */
    double omega, phase;
    long motion_t;             /* t: steps since the motion was set */
    int nthreads;
} orc_sim;

static long node_index(const orc_sim *s, int x, int y, int z) {
    x = ((x % s->nx) + s->nx) % s->nx;
    y = ((y % s->ny) + s->ny) % s->ny;
    z = ((z % s->nz) + s->nz) % s->nz;
    return x + (long)s->nx * (y + (long)s->ny * z);
}
static void node_coords(const orc_sim *s, long n, int *x, int *y, int *z) {
    *x = (int)(n % s->nx);
    *y = (int)((n / s->nx) % s->ny);
    *z = (int)(n / ((long)s->nx * s->ny));
}
static long neighbour(const orc_sim *s, long n, const int e[3], int sign) {
    int x, y, z;
    node_coords(s, n, &x, &y, &z);
    return node_index(s, x + sign * e[0], y + sign * e[1], z + sign * e[2]);
}

orc_sim *orc_create(int dim, int nx, int ny, int nz, int has_h, int has_g,
                    double tau_nu, double tau_D, double tau_eta,
                    const double accel[3], const uint8_t *solid) {
    if (dim != 2 && dim != 3) return NULL;
    if (dim == 2 && nz != 1) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->dim = dim; s->nx = nx; s->ny = ny; s->nz = nz;
    s->has_h = has_h; s->has_g = has_g; s->nB = dim;
    s->N = (long)nx * ny * nz;
    s->tau_nu = tau_nu; s->tau_D = tau_D; s->tau_eta = tau_eta;
    s->nC = has_h ? 1 : 0;
    s->tau_Ds[0] = tau_D;
    for (int k = 0; k < 3; ++k) s->accel[k] = accel ? accel[k] : 0.0;
    s->solid = (uint8_t *)malloc(s->N);
    memcpy(s->solid, solid, s->N);
    int qf = flow_lattice(dim).q, qm = scalar_lattice(dim).q;
    s->f = calloc((size_t)qf * s->N, sizeof(double));
    s->fr = calloc((size_t)qf * s->N, sizeof(double));
    s->fn = calloc((size_t)qf * s->N, sizeof(double));
    if (has_h) {
        s->h = calloc((size_t)qm * s->N, sizeof(double));
        s->hr = calloc((size_t)qm * s->N, sizeof(double));
        s->hn = calloc((size_t)qm * s->N, sizeof(double));
    }
    if (has_g) {
        s->g = calloc((size_t)s->nB * qm * s->N, sizeof(double));
        s->gr = calloc((size_t)s->nB * qm * s->N, sizeof(double));
        s->gn = calloc((size_t)s->nB * qm * s->N, sizeof(double));
    }
    s->rho = calloc(s->N, sizeof(double));
    s->u = calloc(3 * (size_t)s->N, sizeof(double));
    s->C = calloc(s->N, sizeof(double));
    s->B = calloc(3 * (size_t)s->N, sizeof(double));
    s->nbf = malloc(sizeof(int32_t) * qf * s->N);
    s->nbm = malloc(sizeof(int32_t) * qm * s->N);
    lattice L = flow_lattice(dim), M = scalar_lattice(dim);
    for (long n = 0; n < s->N; ++n) {
        for (int a = 0; a < qf; ++a) s->nbf[(long)a * s->N + n] = (int32_t)neighbour(s, n, L.e[a], +1);
        for (int a = 0; a < qm; ++a) s->nbm[(long)a * s->N + n] = (int32_t)neighbour(s, n, M.e[a], +1);
    }
    s->nthreads = 1;
    return s;
}

void orc_destroy(orc_sim *s) {
    if (!s) return;
    free(s->solid); free(s->f); free(s->fr); free(s->fn);
    free(s->h); free(s->hr); free(s->hn); free(s->g); free(s->gr); free(s->gn);
    free(s->rho); free(s->u); free(s->C); free(s->B); free(s->links);
    free(s->nbf); free(s->nbm);
    free(s);
}

void orc_set_threads(orc_sim *s, int n) { s->nthreads = n > 0 ? n : 1; }

/* Several concentration species (call after orc_create with has_h, before
 * the links and the initial state): species k has relaxation time tau_D[k]
 * and initial C0[k] (k >= 1; species 0's initial C is orc_init's C0).
 * Returns 0, or -1 for a bad count or a context without C. */
int orc_set_species(orc_sim *s, int nC, const double *tau_D, const double *C0) {
    if (!s->has_h || nC < 1 || nC > ORC_MAX_SPECIES) return -1;
    for (int k = 0; k < nC; ++k)
        if (!(tau_D[k] > 0.5)) return -1;
    int qm = scalar_lattice(s->dim).q;
    free(s->h); free(s->hr); free(s->hn); free(s->C);
    s->h = calloc((size_t)nC * qm * s->N, sizeof(double));
    s->hr = calloc((size_t)nC * qm * s->N, sizeof(double));
    s->hn = calloc((size_t)nC * qm * s->N, sizeof(double));
    s->C = calloc((size_t)nC * s->N, sizeof(double));
    s->nC = nC;
    for (int k = 0; k < nC; ++k) {
        s->tau_Ds[k] = tau_D[k];
        s->C0s[k] = C0 ? C0[k] : 0.0;
    }
    s->tau_D = tau_D[0];
    return 0;
}

/* The surface reaction network of ORC_REACTION links: n reactions (at most
 * ORC_MAX_REACT), rate[j], order[j * 4 + m] in 0..2 and stoich[j * 4 + i].
 * Returns 0 or -1. */
int orc_set_network(orc_sim *s, int n, const double *rate, const int *order, const double *stoich) {
    if (n < 0 || n > ORC_MAX_REACT) return -1;
    memset(&s->net, 0, sizeof s->net);
    s->net.n = n;
    for (int j = 0; j < n; ++j) {
        s->net.rate[j] = rate[j];
        for (int m = 0; m < ORC_MAX_SPECIES; ++m) {
            if (order[j * ORC_MAX_SPECIES + m] < 0 || order[j * ORC_MAX_SPECIES + m] > 2) return -1;
            s->net.order[j][m] = order[j * ORC_MAX_SPECIES + m];
            s->net.stoich[j][m] = stoich[j * ORC_MAX_SPECIES + m];
        }
    }
    return 0;
}

/* h planes of species k: h[(k * qm + a) * N + n] */
static double *hp(double *h, int qm, long N, int k) { return h + (long)k * qm * N; }

/* g layout: g[(k * qm + a) * N + n] for component k */
static double *gp(double *g, int qm, long N, int k, int a, long n) {
    return &g[((long)k * qm + a) * N + n];
}

/* Validate and store the link list.  Returns 0, or a negative code:
 *  -1 bad field/kind/dir, -2 node not fluid, -3 wall node not solid,
 *  -4 d outside (0,1], -5 duplicate (node, field, dir), -6 an unknown
 *  population without a link. */
int orc_set_links(orc_sim *s, const orc_link *links, long n) {
    int qf = flow_lattice(s->dim).q, qm = scalar_lattice(s->dim).q;
    int nfield = 1 + (s->has_h ? 1 : 0) + (s->has_g ? s->nB : 0);
    (void)nfield;
    /* coverage table: per node, per field slot, per direction */
    int qmax = qf;
    int nslots = ORC_HS1 + ORC_MAX_SPECIES - 1;
    uint8_t *seen = calloc((size_t)s->N * nslots * qmax, 1);
    for (long i = 0; i < n; ++i) {
        const orc_link *lk = &links[i];
        int field = lk->field;
        if (field == ORC_F) {
            if ((lk->kind != ORC_VELOCITY && lk->kind != ORC_VELOCITY_EQ15 && !(lk->kind == ORC_PRESSURE && !s->has_g && !s->has_h))
                || lk->dir <= 0 || lk->dir >= qf) { free(seen); return -1; }
        } else if (species_of(field) >= 0) {
            if (!s->has_h || species_of(field) >= s->nC ||
                (lk->kind != ORC_GIVEN && lk->kind != ORC_FLUX && lk->kind != ORC_NEUMANN_BFL && lk->kind != ORC_FLUX_SIMPLIFIED &&
                 lk->kind != ORC_FLUX_RATIONAL && lk->kind != ORC_REACTION) || lk->dir <= 0 || lk->dir >= qm) { free(seen); return -1; }
        } else if (field >= ORC_G0 && field < ORC_G0 + s->nB) {
            if (!s->has_g || (lk->kind != ORC_GIVEN && lk->kind != ORC_FLUX && lk->kind != ORC_NEUMANN_BFL && lk->kind != ORC_FLUX_SIMPLIFIED) || lk->dir <= 0 || lk->dir >= qm) { free(seen); return -1; }
        } else { free(seen); return -1; }
        if (lk->node < 0 || lk->node >= s->N || s->solid[lk->node]) { free(seen); return -2; }
        lattice L = field == ORC_F ? flow_lattice(s->dim) : scalar_lattice(s->dim);
        long Bn = neighbour(s, lk->node, L.e[lk->dir], -1);
        if (!s->solid[Bn]) { free(seen); return -3; }
        if (!(lk->d > 0.0 && lk->d <= 1.0)) { free(seen); return -4; }
        uint8_t *slot = &seen[((long)lk->node * nslots + field) * qmax + lk->dir];
        if (*slot) { free(seen); return -5; }
        *slot = 1;
    }
    /* completeness: every population arriving from a solid node has a link */
    for (long x = 0; x < s->N; ++x) {
        if (s->solid[x]) continue;
        for (int field = 0; field < nslots; ++field) {
            int sp = species_of(field);
            if (sp >= 0 && sp >= s->nC) continue;
            if (field != ORC_F && sp < 0 && (!s->has_g || field >= ORC_G0 + s->nB)) continue;
            lattice L = field == ORC_F ? flow_lattice(s->dim) : scalar_lattice(s->dim);
            for (int a = 1; a < L.q; ++a) {
                long Bn = neighbour(s, x, L.e[a], -1);
                if (s->solid[Bn] && !seen[((long)x * nslots + field) * qmax + a]) { free(seen); return -6; }
            }
        }
    }
    free(seen);
    free(s->links);
    s->links = malloc(sizeof(orc_link) * (n > 0 ? n : 1));
    memcpy(s->links, links, sizeof(orc_link) * n);
    s->nlinks = n;
    return 0;
}

/* Initial state (R11 reading): populations at equilibrium of the given fields.
 * Any of the arrays may be NULL: rho -> rho0, u -> 0, C -> C0, B -> B0[]. */
void orc_init(orc_sim *s, const double *rho, const double *u, const double *C, const double *B,
              double rho0, double C0, const double B0[3]) {
    s->C0s[0] = C0;
    int qf = flow_lattice(s->dim).q, qm = scalar_lattice(s->dim).q;
    for (long n = 0; n < s->N; ++n) {
        if (s->solid[n]) continue;
        double r = rho ? rho[n] : rho0;
        double uu[3] = {0, 0, 0}, bb[3] = {0, 0, 0};
        if (u) for (int k = 0; k < 3; ++k) uu[k] = u[3 * n + k];
        if (s->has_g) for (int k = 0; k < 3; ++k) bb[k] = B ? B[3 * n + k] : B0[k];
        for (int a = 0; a < qf; ++a)
            s->f[(long)a * s->N + n] = orc_feq(s->dim, a, r, uu, s->has_g ? bb : NULL);
        for (int k = 0; k < s->nC; ++k) {
            double c = (k == 0 && C) ? C[n] : (k == 0 ? C0 : s->C0s[k]);
            for (int a = 0; a < qm; ++a) hp(s->h, qm, s->N, k)[(long)a * s->N + n] = orc_heq(s->dim, a, c, uu);
        }
        if (s->has_g)
            for (int k = 0; k < s->nB; ++k)
                for (int a = 0; a < qm; ++a) *gp(s->g, qm, s->N, k, a, n) = orc_geq(s->dim, a, k, bb, uu);
    }
    s->steps = 0;
}

/* Step 1: moments at t (Eq. 2, 4, 6; body-force shifted velocity per the Guo reading) */
static void compute_moments(orc_sim *s) {
    lattice L = flow_lattice(s->dim), M = scalar_lattice(s->dim);
    long N = s->N;
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->solid[n]) continue;
        double rho = 0, j[3] = {0, 0, 0};
        for (int a = 0; a < L.q; ++a) {
            double fa = s->f[(long)a * N + n];
            rho += fa;
            for (int k = 0; k < 3; ++k) j[k] += L.e[a][k] * fa;
        }
        s->rho[n] = rho;
        for (int k = 0; k < 3; ++k) s->u[3 * n + k] = (j[k] + 0.5 * rho * s->accel[k]) / rho;
        for (int k = 0; k < s->nC; ++k) {
            double C = 0;
            for (int a = 0; a < M.q; ++a) C += hp(s->h, M.q, N, k)[(long)a * N + n];
            s->C[(long)k * N + n] = C;
        }
        if (s->has_g) {
            for (int k = 0; k < 3; ++k) s->B[3 * n + k] = 0.0;
            for (int k = 0; k < s->nB; ++k) {
                double Bk = 0;
                for (int a = 0; a < M.q; ++a) Bk += *gp(s->g, M.q, N, k, a, n);
                s->B[3 * n + k] = Bk;
            }
        }
    }
}

/* Step 2: relaxation (Eq. 1, 3, 5) */
static void relax(orc_sim *s) {
    lattice L = flow_lattice(s->dim), M = scalar_lattice(s->dim);
    long N = s->N;
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->solid[n]) continue;
        double rho = s->rho[n];
        const double *u = &s->u[3 * n];
        const double *B = &s->B[3 * n];
        double F[3] = {rho * s->accel[0], rho * s->accel[1], rho * s->accel[2]};
        for (int a = 0; a < L.q; ++a) {
            double fa = s->f[(long)a * N + n];
            double feq = orc_feq(s->dim, a, rho, u, s->has_g ? B : NULL);
            s->fr[(long)a * N + n] = fa + (feq - fa) / s->tau_nu + orc_guo(s->dim, a, s->tau_nu, u, F);
        }
        for (int k = 0; k < s->nC; ++k) {
            const double *h = hp(s->h, M.q, N, k);
            double *hr = hp(s->hr, M.q, N, k);
            for (int a = 0; a < M.q; ++a) {
                double ha = h[(long)a * N + n];
                hr[(long)a * N + n] = ha + (orc_heq(s->dim, a, s->C[(long)k * N + n], u) - ha) / s->tau_Ds[k];
            }
        }
        if (s->has_g) {
            for (int k = 0; k < s->nB; ++k)
                for (int a = 0; a < M.q; ++a) {
                    double ga = *gp(s->g, M.q, N, k, a, n);
                    *gp(s->gr, M.q, N, k, a, n) = ga + (orc_geq(s->dim, a, k, B, u) - ga) / s->tau_eta;
                }
        }
    }
}

/* Step 3: propagation x -> x + e_a for fluid targets (solid nodes hold zeros) */
static void propagate_field(orc_sim *s, lattice L, const int32_t *nb, const double *pr, double *pn) {
    long N = s->N;
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (long n = 0; n < N; ++n) {
        if (s->solid[n]) {
            for (int a = 0; a < L.q; ++a) pn[(long)a * N + n] = 0.0;
            continue;
        }
        for (int a = 0; a < L.q; ++a) {
            long y = nb[(long)a * N + n];
            if (!s->solid[y]) pn[(long)a * N + y] = pr[(long)a * N + n];
        }
    }
}

/* Gather the inputs of one link from the relaxed populations and moments at t */
static void link_inputs(const orc_sim *s, const orc_link *lk, orc_link *eff, orc_link_in *in) {
    *eff = *lk;
    lattice L = lk->field == ORC_F ? flow_lattice(s->dim) : scalar_lattice(s->dim);
    int a = lk->dir, ap = opposite(L, a);
    long N = s->N, A = lk->node;
    long E = (lk->field == ORC_F ? s->nbf : s->nbm)[(long)a * N + A];   /* E = A + e_a */
    if (s->solid[E]) { E = A; eff->d = 0.5; }       /* E-solid reading */
    const double *pr;
    int sp = species_of(lk->field);
    if (lk->field == ORC_F) pr = s->fr;
    else if (sp >= 0) pr = hp(s->hr, L.q, N, sp);
    else pr = s->gr + (long)(lk->field - ORC_G0) * L.q * N;
    in->p_a_A = pr[(long)a * N + A];
    in->p_ap_A = pr[(long)ap * N + A];
    in->p_ap_E = pr[(long)ap * N + E];
    if (lk->field == ORC_F) { in->phi_A = s->rho[A]; in->phi_E = s->rho[E]; }
    else if (sp >= 0) { in->phi_A = s->C[(long)sp * N + A]; in->phi_E = s->C[(long)sp * N + E]; }
    else {
        int k = lk->field - ORC_G0;
        in->phi_A = s->B[3 * A + k]; in->phi_E = s->B[3 * E + k];
    }
    for (int c = 0; c < 3; ++c) { in->B_A[c] = s->B[3 * A + c]; in->B_E[c] = s->B[3 * E + c]; }
    for (int c = 0; c < 3; ++c) { in->u_A[c] = s->u[3 * A + c]; in->u_E[c] = s->u[3 * E + c]; }
    in->nspecies = s->nC;
    in->net = &s->net;
    for (int m = 0; m < s->nC; ++m) { in->C_A[m] = s->C[(long)m * N + A]; in->C_E[m] = s->C[(long)m * N + E]; }
    if (s->motion && lk->field == ORC_F && (lk->kind == ORC_VELOCITY || lk->kind == ORC_VELOCITY_EQ15)) {
        /* oscillating wall, Eq. 45: the wall velocity of the step t -> t+1 is
         * taken at t, the time of f^eq(X, t) in Eq. 41 and 43 */
        double sc = cos(s->omega * (double)s->motion_t + s->phase);
        for (int c = 0; c < 3; ++c) eff->u_wall[c] = lk->u_wall[c] * sc;
    }
}

/* Step 4: every link sets its unknown population at t+1 */
static void apply_links(orc_sim *s) {
    int qm = scalar_lattice(s->dim).q;
    long N = s->N;
    for (long i = 0; i < s->nlinks; ++i) {
        orc_link eff;
        orc_link_in in;
        link_inputs(s, &s->links[i], &eff, &in);
        double v = orc_eval_link(s->dim, &eff, &in);
        const orc_link *lk = &s->links[i];
        int sp = species_of(lk->field);
        if (lk->field == ORC_F) s->fn[(long)lk->dir * N + lk->node] = v;
        else if (sp >= 0) hp(s->hn, qm, N, sp)[(long)lk->dir * N + lk->node] = v;
        else *gp(s->gn, qm, N, lk->field - ORC_G0, lk->dir, lk->node) = v;
    }
}

void orc_step(orc_sim *s, int nsteps) {
    lattice L = flow_lattice(s->dim), M = scalar_lattice(s->dim);
    for (int it = 0; it < nsteps; ++it) {
        compute_moments(s);
        relax(s);
        propagate_field(s, L, s->nbf, s->fr, s->fn);
        for (int k = 0; k < s->nC; ++k)
            propagate_field(s, M, s->nbm, hp(s->hr, M.q, s->N, k), hp(s->hn, M.q, s->N, k));
        if (s->has_g)
            for (int k = 0; k < s->nB; ++k)
                propagate_field(s, M, s->nbm, s->gr + (long)k * M.q * s->N, s->gn + (long)k * M.q * s->N);
        apply_links(s);
        double *t;
        t = s->f; s->f = s->fn; s->fn = t;
        t = s->h; s->h = s->hn; s->hn = t;
        t = s->g; s->g = s->gn; s->gn = t;
        s->steps++;
        s->motion_t++;
    }
}

/* Moments of the current populations f(t): rho[N], u[3N], C[N], B[3N]; NULL skips.
 * Solid nodes report zeros. */
void orc_moments(orc_sim *s, double *rho, double *u, double *C, double *B) {
    compute_moments(s);
    for (long n = 0; n < s->N; ++n) {
        int sol = s->solid[n];
        if (rho) rho[n] = sol ? 0.0 : s->rho[n];
        if (u) for (int k = 0; k < 3; ++k) u[3 * n + k] = sol ? 0.0 : s->u[3 * n + k];
        if (C) C[n] = (sol || !s->has_h) ? 0.0 : s->C[n];
        if (B) for (int k = 0; k < 3; ++k) B[3 * n + k] = (sol || !s->has_g) ? 0.0 : s->B[3 * n + k];
    }
}

/* Raw population access (tests, checkpoints): which = 0 f, 1 h, 2 g.  Copies
 * q*N (f, h) or nB*q*N (g) doubles. */
long orc_populations(orc_sim *s, int which, double *out, int set) {
    int qf = flow_lattice(s->dim).q, qm = scalar_lattice(s->dim).q;
    double *p = which == 0 ? s->f : which == 1 ? s->h : s->g;
    long cnt = which == 0 ? (long)qf * s->N : which == 1 ? (long)qm * s->N : (long)s->nB * qm * s->N;
    if (!p) return 0;
    if (set) memcpy(p, out, sizeof(double) * cnt);
    else memcpy(out, p, sizeof(double) * cnt);
    return cnt;
}

long orc_steps(const orc_sim *s) { return s->steps; }

/* Oscillating walls (Sec. 5.2, Eq. 45): from now on every velocity link of f
 * uses u_wall * cos(omega * t + phase) in the step from t to t + 1, t counting
 * the steps since this call.  The moving-wall term of flux links
 * of h or g would need the same motion, so a link list holding such a link with
 * a nonzero wall velocity is refused (-1).  Set the links first. */
int orc_set_wall_motion(orc_sim *s, double omega, double phase) {
    for (long i = 0; i < s->nlinks; ++i) {
        const orc_link *lk = &s->links[i];
        if (lk->field != ORC_F && (lk->kind == ORC_FLUX || lk->kind == ORC_FLUX_SIMPLIFIED || lk->kind == ORC_FLUX_RATIONAL ||
                                   lk->kind == ORC_REACTION) &&
            (lk->u_wall[0] != 0.0 || lk->u_wall[1] != 0.0 || lk->u_wall[2] != 0.0))
            return -1;
    }
    s->motion = 1;
    s->omega = omega;
    s->phase = phase;
    s->motion_t = 0;
    return 0;
}

/* FP64 sums over fluid nodes of rho, C and B_k at the current time (reduction row):
 * out[0] = sum rho, out[1] = sum C, out[2..4] = sum B_k, out[5] = number of
 * non-finite populations. */
void orc_sums(orc_sim *s, double out[6]) {
    compute_moments(s);
    for (int i = 0; i < 6; ++i) out[i] = 0.0;
    int qf = flow_lattice(s->dim).q, qm = scalar_lattice(s->dim).q;
    for (long n = 0; n < s->N; ++n) {
        if (s->solid[n]) continue;
        out[0] += s->rho[n];
        if (s->has_h) out[1] += s->C[n];
        if (s->has_g) for (int k = 0; k < 3; ++k) out[2 + k] += s->B[3 * n + k];
        for (int a = 0; a < qf; ++a) if (!isfinite(s->f[(long)a * s->N + n])) out[5] += 1;
        for (int k = 0; k < s->nC; ++k)
            for (int a = 0; a < qm; ++a) if (!isfinite(hp(s->h, qm, s->N, k)[(long)a * s->N + n])) out[5] += 1;
        if (s->has_g) for (int k = 0; k < s->nB; ++k) for (int a = 0; a < qm; ++a)
            if (!isfinite(*gp(s->g, qm, s->N, k, a, n))) out[5] += 1;
    }
}

int orc_sizeof_link(void) { return (int)sizeof(orc_link); }

/* Concentration of species k at the current time (C[N], solid nodes 0) and
 * the FP64 sum over fluid nodes; returns the sum. */
double orc_species(orc_sim *s, int k, double *C) {
    compute_moments(s);
    double sum = 0.0;
    for (long n = 0; n < s->N; ++n) {
        double v = (s->solid[n] || k < 0 || k >= s->nC) ? 0.0 : s->C[(long)k * s->N + n];
        if (C) C[n] = v;
        sum += v;
    }
    return sum;
}

/* The network production rate R_i at given concentrations (tests). */
double orc_network_rate(const orc_sim *s, int i, const double *C) { return network_rate(&s->net, s->nC, i, C); }
