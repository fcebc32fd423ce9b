/*
 * lbrbc_oracle.c -- plain, slow, FP64 CPU oracle of the coupled lattice
 * Boltzmann time step with the general local reactive boundary condition
 * (arXiv 2306.10794, "General local reactive boundary condition for
 * dissolution and precipitation using the lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against a direct,
 * unoptimised statement of the method.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * One time step (Jacobi: every read comes from the state left by the
 * previous step), in the order the paper implies:
 *   1. pull streaming of the flow populations f (Eq. fluid_BGK) and of the
 *      solute populations g (Eq. solute_BGK); halfway bounce-back where the
 *      source node is not active (Sec. 2.1, TRT remark);
 *   2. the reactive boundary condition (Eq. general_RBC with Eqs. k_i_S_Ve,
 *      k_i_S2, k_i_S_New) on the pre-collision populations of every boundary
 *      node, for every link towards a fluid node (wet-node reading);
 *   3. moments (Eqs. fluid_BGK_visc, solute_diffu) and BGK or TRT collision
 *      (Eqs. fluid_BGK, fluid_TRT, solute_BGK, solute_TRT) with the
 *      equilibria of Eqs. fluid_Equilib and solute_equilibrium_function and
 *      the rest-fraction weights of Eqs. RestFraction, RestFractionCs2;
 *   4. the reacted-mass ledger and the solid-fraction update of
 *      Eq. solidFractionUpdate (adjacent growth, Sec. 2.4), with the sign
 *      that conserves mass;
 *   5. phase change at the thresholds phi <= 0 (dissolution) and phi >= 1
 *      (precipitation) with redistribution (Sec. 2.4).
 * Where the paper is silent the reading used is stated next to the code.
 *
 * Compile: gcc -O2 -std=c99 -ffp-contract=off -shared -fPIC -o liblbrbc_oracle.so lbrbc_oracle.c -lm -lpthread
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Parameters (mirrored by ctypes in oracle/__init__.py).              */
/* ------------------------------------------------------------------ */
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_OPEN = 2 };
enum { ORC_NEW = 0, ORC_VERHAEGHE = 1, ORC_PATEL_JU = 2, ORC_ANTIBB = 3 };
enum { ORC_FLUID = 0, ORC_BOUND = 1, ORC_SOLID = 2 };
enum { ORC_KIND_FLUID = 0, ORC_KIND_REACTIVE = 1, ORC_KIND_DIRICHLET = 2 };
enum { ORC_EV_DISSOLVE = 1, ORC_EV_PRECIPITATE = 2 };

typedef struct {
    int dim, nx, ny, nz;
    int flow_q;            /* 19, 9 or 0 (no flow lattice: u = 0)        */
    int solute_q;          /* 7, 5 or 9                                  */
    int bc[3];             /* ORC_PERIODIC / ORC_WALL / ORC_OPEN (x only)*/
    int scheme;            /* ORC_NEW ...                                */
    int phase_change;      /* 0 / 1                                      */
    double tau_flow;       /* tau_NS (BGK) or tau_NS^+ (TRT)             */
    double magic_flow;     /* Lambda; < 0 selects BGK                    */
    double tau_solute;     /* tau_AD (BGK) or tau_AD^+ (TRT): sets D     */
    double magic_solute;   /* Lambda; < 0 selects BGK                    */
    double rest_fraction;  /* J0; < 0 selects the lattice's own weights  */
    double k_r, c_eq, molar_volume;
    double c_init, rho_init;
    double c_dirichlet;    /* concentration held by Dirichlet cells      */
    double c_inlet, u_inlet, rho_outlet;
} orc_params;

/* ------------------------------------------------------------------ */
/* Velocity sets.  D2Q9 and D2Q5 in the order printed in Appendix A    */
/* (Eqs. D2Q9, D2Q5); D3Q19 / D3Q7 are the standard textbook sets.     */
/* ------------------------------------------------------------------ */
typedef struct {
    int q, dim;
    int e[19][3];
    double w[19];
    double cs2;
    int opp[19];
} orc_lat;

static void finish_lattice(orc_lat *L)
{
    for (int i = 0; i < L->q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < L->q; ++j)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] &&
                L->e[j][2] == -L->e[i][2])
                L->opp[i] = j;
    }
}

/* Fill L for lattice (q, dim).  J0 >= 0 applies the rest-fraction method
 * (Eqs. RestFraction, RestFractionCs2), allowed for D2Q5 and D3Q7 only.
 * Returns 0 on success. */
static int make_lattice(orc_lat *L, int q, int dim, double J0)
{
    memset(L, 0, sizeof(*L));
    L->q = q;
    L->dim = dim;
    if (dim == 2 && q == 9) {
        static const int ex[9] = {0, -1, -1, -1, 0, 1, 1, 1, 0};
        static const int ey[9] = {0, 1, 0, -1, -1, -1, 0, 1, 1};
        for (int i = 0; i < 9; ++i) {
            L->e[i][0] = ex[i];
            L->e[i][1] = ey[i];
            if (i == 0) L->w[i] = 4.0 / 9.0;
            else if (ex[i] != 0 && ey[i] != 0) L->w[i] = 1.0 / 36.0;
            else L->w[i] = 1.0 / 9.0;
        }
        L->cs2 = 1.0 / 3.0;
        if (J0 >= 0.0) return 1; /* rest fraction is defined for D2Q5/D3Q7 */
    } else if (dim == 2 && q == 5) {
        static const int ex[5] = {0, -1, 0, 1, 0};
        static const int ey[5] = {0, 0, -1, 0, 1};
        for (int i = 0; i < 5; ++i) {
            L->e[i][0] = ex[i];
            L->e[i][1] = ey[i];
            L->w[i] = (i == 0) ? 1.0 / 3.0 : 1.0 / 6.0;
        }
        L->cs2 = 1.0 / 3.0;
    } else if (dim == 3 && (q == 19 || q == 7)) {
        static const int ex[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        static const int ey[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        static const int ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        for (int i = 0; i < q; ++i) {
            L->e[i][0] = ex[i];
            L->e[i][1] = ey[i];
            L->e[i][2] = ez[i];
        }
        if (q == 19) {
            for (int i = 0; i < 19; ++i)
                L->w[i] = (i == 0) ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            L->cs2 = 1.0 / 3.0;
            if (J0 >= 0.0) return 1;
        } else {
            /* D3Q7 has no printed table; J0 = 1/4 gives the usual weights. */
            if (J0 < 0.0) J0 = 0.25;
        }
    } else {
        return 1;
    }
    if (J0 >= 0.0 && (q == 5 || q == 7)) {
        if (J0 >= 1.0) return 1;
        L->cs2 = (1.0 - J0) / (double)dim;          /* Eq. RestFractionCs2 */
        for (int i = 0; i < q; ++i)
            L->w[i] = (i == 0) ? J0 : L->cs2 / 2.0;   /* Eq. RestFraction    */
    }
    finish_lattice(L);
    return 0;
}

/* Eq. fluid_Equilib. */
static void flow_equilibrium(const orc_lat *L, double rho, const double u[3], double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        double eu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
        feq[i] = L->w[i] * rho *
                 (1.0 + eu / L->cs2 + (eu * eu) / (2.0 * L->cs2 * L->cs2) - uu / (2.0 * L->cs2));
    }
}

/* Eq. solute_equilibrium_function. */
static void solute_equilibrium(const orc_lat *L, double C, const double u[3], double *geq)
{
    for (int i = 0; i < L->q; ++i) {
        double eu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
        geq[i] = C * L->w[i] * (1.0 + eu / L->cs2);
    }
}

/* BGK (Eqs. fluid_BGK, solute_BGK) or TRT (Eqs. fluid_TRT, solute_TRT):
 * the non-equilibrium symmetric part relaxes with 1/tau_sym, the
 * antisymmetric part with 1/tau_anti.  BGK when use_trt == 0 (tau_sym). */
static void collide(const orc_lat *L, double *p, const double *peq, int use_trt,
                    double tau_sym, double tau_anti)
{
    if (!use_trt) {
        for (int i = 0; i < L->q; ++i) p[i] = p[i] - (p[i] - peq[i]) / tau_sym;
        return;
    }
    double out[19];
    for (int i = 0; i < L->q; ++i) {
        int j = L->opp[i];
        double pp = 0.5 * (p[i] + p[j]), pm = 0.5 * (p[i] - p[j]);       /* Eq. fluid_TRT_terms */
        double ep = 0.5 * (peq[i] + peq[j]), em = 0.5 * (peq[i] - peq[j]);
        out[i] = p[i] - (pp - ep) / tau_sym - (pm - em) / tau_anti;
    }
    for (int i = 0; i < L->q; ++i) p[i] = out[i];
}

/* Eq. general_RBC for a finite k; the anti-bounce-back limit otherwise. */
static double rbc_value(double k, double w, double c_eq, double gt, int infinite)
{
    if (infinite) return 2.0 * w * c_eq - gt;
    return k / (1.0 + k) * 2.0 * w * c_eq + (1.0 - k) / (1.0 + k) * gt;
}

/* ------------------------------------------------------------------ */
/* Simulation state.                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    orc_params p;
    orc_lat LF, LG, LN;  /* flow, solute, normal-estimation lattice */
    long N;
    int has_flow;
    unsigned char *kind, *cls;
    double *fpost, *gpost, *fnew, *gnew;
    double *phi, *kfield, *inlet_ux, *normal;
    unsigned char *normal_ok;
    double *M;              /* per-node reacted mass of this step       */
    double *mlink;          /* per-node, per-direction ledger (solute q) */
    double *C, *rho;        /* per-node moments of this step            */
    double *usol;           /* per-node velocity the solute collision used (3N) */
    double unpaid, dirichlet_in, open_in, reacted_total;
    long step;
    int nthreads;           /* z-slabs of the per-cell loop (timing only)  */
    long nev, capev;
    long *ev_step, *ev_node;
    int *ev_kind;
} orc_sim;

#define IDX(s, x, y, z) ((long)(x) + (long)(s)->p.nx * ((long)(y) + (long)(s)->p.ny * (long)(z)))

enum { NB_IN = 0, NB_WALL = 1, NB_INLET = 2, NB_OUTLET = 3 };

/* Neighbour of (x,y,z) displaced by d.  A link leaving through the x faces
 * of an open x axis is an inlet (x < 0) or outlet (x >= nx) link whatever its
 * other components; otherwise a coordinate outside a wall axis is a wall. */
static int neighbour(const orc_sim *s, int x, int y, int z, const int d[3], long *out)
{
    int c[3] = {x + d[0], y + d[1], z + d[2]};
    int n[3] = {s->p.nx, s->p.ny, s->p.nz};
    if (s->p.bc[0] == ORC_OPEN) {
        if (c[0] < 0) return NB_INLET;
        if (c[0] >= n[0]) return NB_OUTLET;
    }
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (s->p.bc[a] == ORC_PERIODIC) c[a] = ((c[a] % n[a]) + n[a]) % n[a];
            else return NB_WALL;
        }
    }
    *out = IDX(s, c[0], c[1], c[2]);
    return NB_IN;
}

/* Solid indicator used by the wall-normal estimate: 1 for solid cells and
 * for positions beyond a wall axis; open axes are extended by clamping. */
static double solid_indicator(const orc_sim *s, const unsigned char *kind, int x, int y, int z, const int d[3])
{
    int c[3] = {x + d[0], y + d[1], z + d[2]};
    int n[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (s->p.bc[a] == ORC_PERIODIC) c[a] = ((c[a] % n[a]) + n[a]) % n[a];
            else if (s->p.bc[a] == ORC_OPEN) c[a] = c[a] < 0 ? 0 : n[a] - 1;
            else return 1.0;
        }
    }
    return kind[IDX(s, c[0], c[1], c[2])] != ORC_KIND_FLUID ? 1.0 : 0.0;
}

/* Node classes from the cell kinds: a solid cell with at least one fluid
 * neighbour along the solute lattice is a (wet) boundary node. */
static void classify(orc_sim *s, const unsigned char *kind, unsigned char *cls)
{
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long id = IDX(s, x, y, z);
                if (kind[id] == ORC_KIND_FLUID) { cls[id] = ORC_FLUID; continue; }
                int wet = 0;
                for (int i = 1; i < s->LG.q; ++i) {
                    long nb;
                    if (neighbour(s, x, y, z, s->LG.e[i], &nb) == NB_IN && kind[nb] == ORC_KIND_FLUID) wet = 1;
                }
                cls[id] = wet ? ORC_BOUND : ORC_SOLID;
            }
}

/* Wall normal by the isotropic finite-difference gradient of the solid
 * indicator (Sec. 3.2 names the method): grad s = cs^-2 sum_i w_i s(x+e_i) e_i
 * over D2Q9 / D3Q19; n = -grad s / |grad s| points from solid into fluid.
 * The sum is evaluated exactly: with the integer weights 36 w_i it is an
 * integer vector proportional to grad s, so components that vanish by
 * symmetry are exactly zero (the split of the precipitation excess, Sec. 2.4,
 * changes discontinuously when sum (e_o . n)_+ reaches zero). */
static void compute_normals(orc_sim *s)
{
    const orc_lat *L = &s->LN;
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long id = IDX(s, x, y, z);
                long gi[3] = {0, 0, 0};
                s->normal_ok[id] = 0;
                s->normal[3 * id] = s->normal[3 * id + 1] = s->normal[3 * id + 2] = 0.0;
                if (s->cls[id] != ORC_BOUND) continue;
                for (int i = 1; i < L->q; ++i) {
                    long wi = lround(36.0 * L->w[i]);
                    long si = (long)solid_indicator(s, s->kind, x, y, z, L->e[i]);
                    for (int a = 0; a < 3; ++a) gi[a] += wi * si * L->e[i][a];
                }
                if (gi[0] == 0 && gi[1] == 0 && gi[2] == 0) continue;
                double len = sqrt((double)(gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]));
                for (int a = 0; a < 3; ++a) s->normal[3 * id + a] = -(double)gi[a] / len;
                s->normal_ok[id] = 1;
            }
}

/* Projection (e_o . n)_+ of a reflected direction onto the wall normal; a
 * cell whose normal is undefined treats every link as aligned (1). */
static double kappa(const orc_sim *s, long id, const int e[3])
{
    if (!s->normal_ok[id]) return 1.0;
    double d = e[0] * s->normal[3 * id] + e[1] * s->normal[3 * id + 1] + e[2] * s->normal[3 * id + 2];
    return d > 0.0 ? d : 0.0;
}

static double tau_other(double tau, double magic) { return 0.5 + magic / (tau - 0.5); }

static void log_event(orc_sim *s, long node, int kind)
{
    if (s->nev == s->capev) {
        s->capev = s->capev ? 2 * s->capev : 256;
        s->ev_step = (long *)realloc(s->ev_step, s->capev * sizeof(long));
        s->ev_node = (long *)realloc(s->ev_node, s->capev * sizeof(long));
        s->ev_kind = (int *)realloc(s->ev_kind, s->capev * sizeof(int));
    }
    s->ev_step[s->nev] = s->step;
    s->ev_node[s->nev] = node;
    s->ev_kind[s->nev] = kind;
    s->nev++;
}

/* ------------------------------------------------------------------ */
/* Creation                                                            */
/* ------------------------------------------------------------------ */
void orc_destroy(void *h);

void *orc_create(const orc_params *p, const unsigned char *mask, const double *kfield,
                 const double *c_init, const double *u_init, const double *phi_init,
                 const double *inlet_ux)
{
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    if (p->dim == 2) s->p.nz = 1;
    s->N = (long)s->p.nx * s->p.ny * s->p.nz;
    s->has_flow = p->flow_q != 0;
    if (make_lattice(&s->LG, p->solute_q, p->dim, p->rest_fraction)) { free(s); return NULL; }
    if (s->has_flow && make_lattice(&s->LF, p->flow_q, p->dim, -1.0)) { free(s); return NULL; }
    make_lattice(&s->LN, p->dim == 2 ? 9 : 19, p->dim, -1.0);
    long N = s->N;
    int qf = s->has_flow ? s->LF.q : 1, qg = s->LG.q;
    s->kind = (unsigned char *)calloc(N, 1);
    s->cls = (unsigned char *)calloc(N, 1);
    s->fpost = (double *)calloc((size_t)qf * N, sizeof(double));
    s->fnew = (double *)calloc((size_t)qf * N, sizeof(double));
    s->gpost = (double *)calloc((size_t)qg * N, sizeof(double));
    s->gnew = (double *)calloc((size_t)qg * N, sizeof(double));
    s->phi = (double *)calloc(N, sizeof(double));
    s->normal = (double *)calloc(3 * N, sizeof(double));
    s->normal_ok = (unsigned char *)calloc(N, 1);
    s->M = (double *)calloc(N, sizeof(double));
    s->mlink = (double *)calloc((size_t)qg * N, sizeof(double));
    s->C = (double *)calloc(N, sizeof(double));
    s->rho = (double *)calloc(N, sizeof(double));
    s->usol = (double *)calloc(3 * N, sizeof(double));
    s->inlet_ux = (double *)calloc((size_t)s->p.ny * s->p.nz, sizeof(double));
    for (long i = 0; i < (long)s->p.ny * s->p.nz; ++i) s->inlet_ux[i] = inlet_ux ? inlet_ux[i] : p->u_inlet;
    if (kfield) {
        s->kfield = (double *)malloc(N * sizeof(double));
        memcpy(s->kfield, kfield, N * sizeof(double));
    }
    for (long i = 0; i < N; ++i) s->kind[i] = mask[i];
    classify(s, s->kind, s->cls);
    compute_normals(s);
    for (long id = 0; id < N; ++id) {
        double u[3] = {0, 0, 0};
        if (u_init && s->cls[id] == ORC_FLUID) { u[0] = u_init[3 * id]; u[1] = u_init[3 * id + 1]; u[2] = u_init[3 * id + 2]; }
        double C = c_init ? c_init[id] : (s->kind[id] == ORC_KIND_DIRICHLET ? p->c_dirichlet : p->c_init);
        double feq[19], geq[19];
        if (s->cls[id] == ORC_FLUID && s->has_flow) {
            flow_equilibrium(&s->LF, p->rho_init, u, feq);
            for (int i = 0; i < s->LF.q; ++i) s->fpost[i * N + id] = feq[i];
        }
        if (s->cls[id] != ORC_SOLID) {
            solute_equilibrium(&s->LG, C, u, geq);
            for (int i = 0; i < qg; ++i) s->gpost[i * N + id] = geq[i];
        }
        if (phi_init) s->phi[id] = phi_init[id];
        else s->phi[id] = s->kind[id] == ORC_KIND_REACTIVE ? 1.0 : 0.0;
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Phase change (Sec. 2.4), simultaneous for all cells that crossed a  */
/* threshold in this step.                                             */
/* ------------------------------------------------------------------ */
static void phase_change(orc_sim *s)
{
    long N = s->N;
    const orc_lat *G = &s->LG;
    int qg = G->q, qf = s->has_flow ? s->LF.q : 1;
    double Vm = s->p.molar_volume;
    unsigned char *ev = (unsigned char *)calloc(N, 1);
    long count = 0;
    for (long id = 0; id < N; ++id) {
        if (s->cls[id] == ORC_BOUND && s->kind[id] == ORC_KIND_REACTIVE && s->phi[id] <= 0.0) { ev[id] = ORC_EV_DISSOLVE; count++; }
        if (s->cls[id] == ORC_FLUID && s->phi[id] >= 1.0) { ev[id] = ORC_EV_PRECIPITATE; count++; }
    }
    if (!count) { free(ev); return; }

    /* New kinds, classes and normals. */
    unsigned char *kind2 = (unsigned char *)malloc(N), *cls2 = (unsigned char *)malloc(N);
    for (long id = 0; id < N; ++id) {
        kind2[id] = s->kind[id];
        if (ev[id] == ORC_EV_DISSOLVE) kind2[id] = ORC_KIND_FLUID;
        if (ev[id] == ORC_EV_PRECIPITATE) kind2[id] = ORC_KIND_REACTIVE;
    }
    classify(s, kind2, cls2);
    unsigned char *kind_old = s->kind, *cls_old = s->cls;
    s->kind = kind2;
    s->cls = cls2;
    compute_normals(s); /* post-event normals (needed for the excess weights) */

    double *phi2 = (double *)malloc(N * sizeof(double));
    memcpy(phi2, s->phi, N * sizeof(double));
    double *g2 = s->gnew, *f2 = s->fnew; /* post-collision state, edited in place below */
    double *g_pre = (double *)malloc((size_t)qg * N * sizeof(double));
    memcpy(g_pre, g2, (size_t)qg * N * sizeof(double));
    double *cinit_of = (double *)calloc(N, sizeof(double));

    /* (a) states of the event cells themselves */
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long id = IDX(s, x, y, z);
                if (ev[id] == ORC_EV_DISSOLVE) {
                    /* initial concentration: mean over the (pre-event) fluid neighbours */
                    double sc = 0.0, sr = 0.0;
                    int nf = 0;
                    for (int i = 1; i < qg; ++i) {
                        long nb;
                        if (neighbour(s, x, y, z, G->e[i], &nb) == NB_IN && cls_old[nb] == ORC_FLUID) {
                            sc += s->C[nb];
                            sr += s->rho[nb];
                            nf++;
                        }
                    }
                    double cinit = nf ? sc / nf : s->C[id];
                    double rinit = nf ? sr / nf : s->p.rho_init;
                    cinit_of[id] = cinit;
                    for (int i = 0; i < qg; ++i) g2[i * N + id] = G->w[i] * cinit;
                    if (s->has_flow)
                        for (int i = 0; i < qf; ++i) f2[i * N + id] = s->LF.w[i] * rinit;
                    phi2[id] = 0.0;
                    log_event(s, id, ORC_EV_DISSOLVE);
                } else if (ev[id] == ORC_EV_PRECIPITATE) {
                    double phic = s->phi[id] + Vm * s->C[id];
                    int nf = 0;
                    for (int i = 1; i < qg; ++i) {
                        long nb;
                        if (neighbour(s, x, y, z, G->e[i], &nb) == NB_IN && kind2[nb] == ORC_KIND_FLUID) nf++;
                    }
                    phi2[id] = nf ? 1.0 : phic;
                    for (int i = 0; i < qg; ++i) g2[i * N + id] = 0.0;
                    if (s->has_flow)
                        for (int i = 0; i < qf; ++i) f2[i * N + id] = 0.0;
                    log_event(s, id, ORC_EV_PRECIPITATE);
                }
            }

    /* (b) charges of dissolution to the post-event solid neighbours and the
     *     precipitation excess to the post-event fluid neighbours */
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long id = IDX(s, x, y, z);
                if (ev[id] == ORC_EV_DISSOLVE) {
                    /* charge = V_m (C_init - C_b) - phi_b: the solute given to the
                     * new fluid cell plus the overshoot below phi = 0 */
                    double Q = Vm * (cinit_of[id] - s->C[id]) - s->phi[id];
                    int ns = 0;
                    long nbs[19];
                    for (int i = 1; i < qg; ++i) {
                        long nb;
                        if (neighbour(s, x, y, z, G->e[i], &nb) == NB_IN && kind2[nb] == ORC_KIND_REACTIVE) nbs[ns++] = nb;
                    }
                    if (ns) for (int k = 0; k < ns; ++k) phi2[nbs[k]] -= Q / ns;
                    else s->unpaid -= Q / Vm;
                } else if (ev[id] == ORC_EV_PRECIPITATE) {
                    double excess = s->phi[id] + Vm * s->C[id] - 1.0;
                    int nf = 0;
                    long nbs[19];
                    double wk[19], sk = 0.0;
                    for (int i = 1; i < qg; ++i) {
                        long nb;
                        if (neighbour(s, x, y, z, G->e[i], &nb) == NB_IN && kind2[nb] == ORC_KIND_FLUID) {
                            nbs[nf] = nb;
                            wk[nf] = kappa(s, id, G->e[i]);
                            sk += wk[nf];
                            nf++;
                        }
                    }
                    for (int k = 0; k < nf; ++k) {
                        double share = sk > 0.0 ? wk[k] / sk : 1.0 / nf;
                        double dC = excess / Vm * share;
                        for (int i = 0; i < qg; ++i) g2[i * N + nbs[k]] += G->w[i] * dC;
                    }
                }
            }

    /* (c) cells whose class changed without an event of their own */
    for (long id = 0; id < N; ++id) {
        if (ev[id]) continue;
        if (cls_old[id] == ORC_BOUND && s->cls[id] == ORC_SOLID) {
            double C = 0.0;
            for (int i = 0; i < qg; ++i) C += g_pre[i * N + id];
            if (s->kind[id] == ORC_KIND_REACTIVE) phi2[id] += Vm * C;
            else s->dirichlet_in -= C;
            for (int i = 0; i < qg; ++i) g2[i * N + id] = 0.0;
        } else if (cls_old[id] == ORC_SOLID && s->cls[id] == ORC_BOUND) {
            for (int i = 0; i < qg; ++i) g2[i * N + id] = 0.0;
        }
    }
    memcpy(s->phi, phi2, N * sizeof(double));
    free(phi2);
    free(g_pre);
    free(cinit_of);
    free(kind_old);
    free(cls_old);
    free(ev);
}

/* ------------------------------------------------------------------ */
/* One time step                                                       */
/* ------------------------------------------------------------------ */
/* Accumulators of the ledger terms summed over cells. */
typedef struct {
    double *open_in, *dirichlet_in, *reacted;
} orc_acc;

/* Steps 1-4 of one time step (streaming, reactive boundary condition,
 * moments, collision, per-cell ledger) for the cells with z0 <= z < z1. */
static void cells_slab(orc_sim *s, int z0, int z1, orc_acc acc)
{
    const orc_params *p = &s->p;
    long N = s->N;
    const orc_lat *F = &s->LF, *G = &s->LG;
    int qf = s->has_flow ? F->q : 0, qg = G->q;
    int trt_f = p->magic_flow >= 0.0, trt_g = p->magic_solute >= 0.0;
    double tf_sym = p->tau_flow, tf_anti = trt_f ? tau_other(p->tau_flow, p->magic_flow) : p->tau_flow;
    /* solute TRT: the tau that sets D relaxes the antisymmetric part (Eq. solute_TRT) */
    double tg_anti = p->tau_solute, tg_sym = trt_g ? tau_other(p->tau_solute, p->magic_solute) : p->tau_solute;
    double gamma = p->tau_solute / (p->tau_solute - 0.5);

    for (int z = z0; z < z1; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long id = IDX(s, x, y, z);
                s->M[id] = 0.0;
                for (int i = 0; i < qg; ++i) s->mlink[i * N + id] = 0.0;
                if (s->cls[id] == ORC_SOLID) {
                    s->C[id] = 0.0;
                    s->rho[id] = 0.0;
                    continue;
                }
                double u[3] = {0, 0, 0}, rho = 0.0;

                /* ---- flow lattice (fluid nodes only) ---- */
                if (s->cls[id] == ORC_FLUID && qf) {
                    double f[19], feq[19];
                    double uo[3] = {0, 0, 0}, ro = 0.0; /* previous-step velocity for the outlet */
                    for (int i = 0; i < qf; ++i) {
                        ro += s->fpost[i * N + id];
                        for (int a = 0; a < 3; ++a) uo[a] += s->fpost[i * N + id] * F->e[i][a];
                    }
                    for (int a = 0; a < 3; ++a) uo[a] /= ro;
                    double uo2 = uo[0] * uo[0] + uo[1] * uo[1] + uo[2] * uo[2];
                    for (int i = 0; i < qf; ++i) {
                        int me[3] = {-F->e[i][0], -F->e[i][1], -F->e[i][2]};
                        long src;
                        int st = neighbour(s, x, y, z, me, &src);
                        double bb = s->fpost[F->opp[i] * N + id];
                        if (st == NB_IN && s->cls[src] == ORC_FLUID) f[i] = s->fpost[i * N + src];
                        else if (st == NB_INLET) {
                            /* moving-wall bounce-back with the inlet velocity */
                            double eu = F->e[i][0] * s->inlet_ux[y + p->ny * z];
                            f[i] = bb + 2.0 * F->w[i] * 1.0 * eu / F->cs2;
                        } else if (st == NB_OUTLET) {
                            /* pressure anti-bounce-back at rho_outlet */
                            double eu = F->e[i][0] * uo[0] + F->e[i][1] * uo[1] + F->e[i][2] * uo[2];
                            f[i] = -bb + 2.0 * F->w[i] * p->rho_outlet *
                                             (1.0 + eu * eu / (2.0 * F->cs2 * F->cs2) - uo2 / (2.0 * F->cs2));
                        } else f[i] = bb; /* halfway bounce-back */
                    }
                    for (int i = 0; i < qf; ++i) {
                        rho += f[i];
                        for (int a = 0; a < 3; ++a) u[a] += f[i] * F->e[i][a];
                    }
                    for (int a = 0; a < 3; ++a) u[a] /= rho;
                    flow_equilibrium(F, rho, u, feq);
                    collide(F, f, feq, trt_f, tf_sym, tf_anti);
                    for (int i = 0; i < qf; ++i) s->fnew[i * N + id] = f[i];
                }
                s->rho[id] = rho;

                /* ---- solute lattice (fluid and boundary nodes) ---- */
                double g[19], geq[19], g_pre[19];
                double Cold = 0.0;
                for (int i = 0; i < qg; ++i) Cold += s->gpost[i * N + id];
                for (int i = 0; i < qg; ++i) {
                    int me[3] = {-G->e[i][0], -G->e[i][1], -G->e[i][2]};
                    long src;
                    int st = neighbour(s, x, y, z, me, &src);
                    double bb = s->gpost[G->opp[i] * N + id];
                    if (st == NB_IN && s->cls[src] != ORC_SOLID) g[i] = s->gpost[i * N + src];
                    else if (st == NB_INLET && s->cls[id] == ORC_FLUID) {
                        g[i] = -bb + 2.0 * G->w[i] * p->c_inlet;   /* anti-bounce-back, C = c_inlet */
                        *acc.open_in += g[i] - bb;
                    } else if (st == NB_OUTLET && s->cls[id] == ORC_FLUID) {
                        g[i] = -bb + 2.0 * G->w[i] * Cold;        /* zero-gradient outlet */
                        *acc.open_in += g[i] - bb;
                    } else g[i] = bb;
                }
                if (s->cls[id] == ORC_BOUND) {
                    /* Eq. general_RBC on every link towards a fluid node, all
                     * links evaluated from the streamed (pre-RBC) values. */
                    for (int i = 0; i < qg; ++i) g_pre[i] = g[i];
                    double kr = s->kfield ? s->kfield[id] : p->k_r;
                    for (int o = 1; o < qg; ++o) {
                        long nb;
                        if (neighbour(s, x, y, z, G->e[o], &nb) != NB_IN || s->cls[nb] != ORC_FLUID) continue;
                        double gt = g_pre[G->opp[o]];
                        double val;
                        if (s->kind[id] == ORC_KIND_DIRICHLET) {
                            val = rbc_value(0.0, G->w[o], p->c_dirichlet, gt, 1);
                        } else {
                            double kap = kappa(s, id, G->e[o]);
                            double k = 0.0;
                            int inf = 0;
                            switch (p->scheme) {
                            case ORC_NEW: k = gamma * kr * kap / G->cs2; break;        /* Eq. k_i_S_New */
                            case ORC_VERHAEGHE: k = kr * kap / G->cs2; break;          /* Eq. k_i_S_Ve  */
                            case ORC_PATEL_JU:                                        /* Eq. k_i_S2    */
                                if (kap > 0.0) k = gamma * kr / (G->cs2 * kap);
                                else inf = 1;
                                break;
                            default: inf = 1; break;                                  /* anti-BB      */
                            }
                            /* a cell with k_r = 0 does not react under any scheme: the
                             * anti-bounce-back limit is the k_r -> infinity limit of a
                             * reacting cell, and k_r / (e.n) is 0 for k_r = 0 */
                            if (kr == 0.0) { k = 0.0; inf = 0; }
                            val = rbc_value(k, G->w[o], p->c_eq, gt, inf);
                        }
                        s->mlink[o * N + id] = val - g_pre[o];
                        g[o] = val;
                    }
                    double Msum = 0.0;
                    for (int o = 1; o < qg; ++o) Msum += s->mlink[o * N + id];
                    if (s->kind[id] == ORC_KIND_DIRICHLET) *acc.dirichlet_in += Msum;
                    else {
                        s->M[id] = Msum;
                        *acc.reacted += Msum;
                    }
                    u[0] = u[1] = u[2] = 0.0;
                }
                double C = 0.0;
                for (int i = 0; i < qg; ++i) C += g[i];
                s->C[id] = C;
                for (int a = 0; a < 3; ++a) s->usol[3 * id + a] = u[a];
                solute_equilibrium(G, C, u, geq);
                collide(G, g, geq, trt_g, tg_sym, tg_anti);
                for (int i = 0; i < qg; ++i) s->gnew[i * N + id] = g[i];
            }

}

/* The per-cell loop may run as z-slabs on several host threads (used only to
 * time the oracle on all cores): every cell reads the previous step's state
 * and writes only its own entries, and each slab sums its ledger terms in
 * its own accumulators, added in slab order afterwards.  With one thread the
 * loop and its sums are exactly the single-slab loop above. */
typedef struct {
    orc_sim *s;
    int z0, z1;
    double open_in, dirichlet_in, reacted;
} orc_slab;

static void *slab_main(void *arg)
{
    orc_slab *a = (orc_slab *)arg;
    orc_acc acc = {&a->open_in, &a->dirichlet_in, &a->reacted};
    cells_slab(a->s, a->z0, a->z1, acc);
    return NULL;
}

static void cells_all(orc_sim *s)
{
    int nt = s->nthreads > 1 ? s->nthreads : 1;
    if (nt > s->p.nz) nt = s->p.nz;
    if (nt <= 1) {
        orc_acc acc = {&s->open_in, &s->dirichlet_in, &s->reacted_total};
        cells_slab(s, 0, s->p.nz, acc);
        return;
    }
    orc_slab *sl = (orc_slab *)calloc(nt, sizeof(orc_slab));
    pthread_t *th = (pthread_t *)calloc(nt, sizeof(pthread_t));
    for (int t = 0; t < nt; ++t) {
        sl[t].s = s;
        sl[t].z0 = (int)((long)s->p.nz * t / nt);
        sl[t].z1 = (int)((long)s->p.nz * (t + 1) / nt);
        pthread_create(&th[t], NULL, slab_main, &sl[t]);
    }
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    for (int t = 0; t < nt; ++t) {
        s->open_in += sl[t].open_in;
        s->dirichlet_in += sl[t].dirichlet_in;
        s->reacted_total += sl[t].reacted;
    }
    free(sl);
    free(th);
}

static void one_step(orc_sim *s)
{
    const orc_params *p = &s->p;
    long N = s->N;
    const orc_lat *G = &s->LG;
    int qg = G->q;

    cells_all(s);

    /* Eq. solidFractionUpdate, adjacent growth: dissolution lowers phi of the
     * boundary cell; precipitation raises phi of the fluid cells at the ends of
     * its links in proportion to |m_l|.  Sign chosen so that
     * sum C + sum phi / V_m is conserved. */
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long id = IDX(s, x, y, z);
                if (s->cls[id] != ORC_BOUND || s->kind[id] != ORC_KIND_REACTIVE) continue;
                double Mb = s->M[id];
                if (Mb > 0.0) s->phi[id] -= p->molar_volume * Mb;
                else if (Mb < 0.0) {
                    double S = 0.0;
                    for (int o = 1; o < qg; ++o) S += fabs(s->mlink[o * N + id]);
                    for (int o = 1; o < qg; ++o) {
                        double m = s->mlink[o * N + id];
                        if (m == 0.0) continue;
                        long nb;
                        if (neighbour(s, x, y, z, G->e[o], &nb) != NB_IN) continue;
                        s->phi[nb] += -p->molar_volume * Mb * fabs(m) / S;
                    }
                }
            }

    if (p->phase_change) phase_change(s);

    double *t;
    t = s->fpost; s->fpost = s->fnew; s->fnew = t;
    t = s->gpost; s->gpost = s->gnew; s->gnew = t;
    s->step++;
}

/* Number of host threads of the per-cell loop (1: the plain loop). */
void orc_set_threads(void *h, int n)
{
    ((orc_sim *)h)->nthreads = n < 1 ? 1 : n;
}

int orc_step(void *h, long n)
{
    orc_sim *s = (orc_sim *)h;
    for (long k = 0; k < n; ++k) one_step(s);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Outputs                                                             */
/* ------------------------------------------------------------------ */
/* Moments of the current (post-collision) state: u and rho of fluid cells,
 * C of active cells, phi of all cells.  Inactive entries are 0. */
void orc_fields(void *h, double *u, double *rho, double *c, double *phi)
{
    orc_sim *s = (orc_sim *)h;
    long N = s->N;
    for (long id = 0; id < N; ++id) {
        double r = 0.0, m[3] = {0, 0, 0}, C = 0.0;
        if (s->cls[id] == ORC_FLUID && s->has_flow) {
            for (int i = 0; i < s->LF.q; ++i) {
                r += s->fpost[i * N + id];
                for (int a = 0; a < 3; ++a) m[a] += s->fpost[i * N + id] * s->LF.e[i][a];
            }
            for (int a = 0; a < 3; ++a) m[a] /= r;
        }
        if (s->cls[id] != ORC_SOLID)
            for (int i = 0; i < s->LG.q; ++i) C += s->gpost[i * N + id];
        if (u) for (int a = 0; a < 3; ++a) u[3 * id + a] = m[a];
        if (rho) rho[id] = r;
        if (c) c[id] = C;
        if (phi) phi[id] = s->phi[id];
    }
}

void orc_classes(void *h, unsigned char *cls)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(cls, s->cls, s->N);
}

void orc_normals(void *h, double *n)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(n, s->normal, 3 * s->N * sizeof(double));
}

/* [0] sum of C over active cells, [1] sum of phi / V_m over all cells,
 * [2] unpaid dissolution charge, [3] cumulative Dirichlet-cell inflow,
 * [4] cumulative open-boundary inflow, [5] cumulative reacted mass,
 * [6] step counter. */
void orc_ledger(void *h, double *out)
{
    orc_sim *s = (orc_sim *)h;
    double sc = 0.0, sp = 0.0;
    for (long id = 0; id < s->N; ++id) {
        if (s->cls[id] != ORC_SOLID)
            for (int i = 0; i < s->LG.q; ++i) sc += s->gpost[i * s->N + id];
        sp += s->phi[id];
    }
    out[0] = sc;
    out[1] = sp / s->p.molar_volume;
    out[2] = s->unpaid;
    out[3] = s->dirichlet_in;
    out[4] = s->open_in;
    out[5] = s->reacted_total;
    out[6] = (double)s->step;
}

/* Reacted mass M_b of every boundary cell in the last step (0 elsewhere). */
void orc_reacted(void *h, double *M)
{
    orc_sim *s = (orc_sim *)h;
    memcpy(M, s->M, s->N * sizeof(double));
}

long orc_event_count(void *h) { return ((orc_sim *)h)->nev; }

void orc_events(void *h, long *step, long *node, int *kind)
{
    orc_sim *s = (orc_sim *)h;
    for (long i = 0; i < s->nev; ++i) {
        step[i] = s->ev_step[i];
        node[i] = s->ev_node[i];
        kind[i] = s->ev_kind[i];
    }
}

void orc_destroy(void *h)
{
    orc_sim *s = (orc_sim *)h;
    if (!s) return;
    free(s->kind); free(s->cls); free(s->fpost); free(s->gpost); free(s->fnew); free(s->gnew);
    free(s->phi); free(s->kfield); free(s->inlet_ux); free(s->normal); free(s->normal_ok);
    free(s->M); free(s->mlink); free(s->C); free(s->rho); free(s->usol);
    free(s->ev_step); free(s->ev_node); free(s->ev_kind);
    free(s);
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of the reacted mass (an extension: the paper has   */
/* no gradient).                                                       */
/* ------------------------------------------------------------------ */
/* With phase change off and the flow independent of k_r and c_eq, one
 * solute step maps the post-collision populations g affinely to the next
 * ones:  h = pull(g) with the bounce-back and open-boundary rules (steps 1-2
 * of the step above), h' = Eq. general_RBC on the links of boundary cells,
 * g_new = collide(h') with the velocity u that step used, and the reacted
 * mass grows by the ledger sum of (h'_o - h_o) over reactive links.  The
 * adjoint below runs the forward steps, keeping g and u of every step, then
 * walks back: lambda (dJ / d g of the later state) is pulled back through
 * each stage by the transpose of that stage, written as the scatter of the
 * stage's own gather, and the derivative of h'_o with respect to k and c_eq
 * is collected on the way.  The collision matrix of a cell is taken by
 * applying the oracle's own collide() to unit vectors (it is linear in h'
 * for a fixed u).  Cells with k_r = 0 reflect without reacting under every
 * scheme (as in the forward step), so they take no part in the k_r
 * gradients.  Memory: (q + 3) N doubles per step. */

/* k of a reactive link of cell id towards direction o and dk/dk_r; inf = 1
 * for the anti-bounce-back limit (no k dependence). */
static void link_k(const orc_sim *s, long id, int o, double kr, double *k, double *dkdkr, int *inf)
{
    const orc_lat *G = &s->LG;
    double gamma = s->p.tau_solute / (s->p.tau_solute - 0.5);
    double kap = kappa(s, id, G->e[o]);
    *k = 0.0;
    *dkdkr = 0.0;
    *inf = 0;
    switch (s->p.scheme) {
    case ORC_NEW: *dkdkr = gamma * kap / G->cs2; break;
    case ORC_VERHAEGHE: *dkdkr = kap / G->cs2; break;
    case ORC_PATEL_JU:
        if (kap > 0.0) *dkdkr = gamma / (G->cs2 * kap);
        else *inf = 1;
        break;
    default: *inf = 1; break;
    }
    *k = *dkdkr * kr;
}

int orc_adjoint(void *h, long n, double *J, double *dJ_dk, double *dJ_dceq, double *dJ_dkfield)
{
    orc_sim *s = (orc_sim *)h;
    if (s->p.phase_change || n < 1) return 1;
    const orc_params *p = &s->p;
    const orc_lat *G = &s->LG;
    long N = s->N;
    int qg = G->q;
    int trt_g = p->magic_solute >= 0.0;
    double tg_anti = p->tau_solute, tg_sym = trt_g ? tau_other(p->tau_solute, p->magic_solute) : p->tau_solute;
    double *gs = (double *)malloc((size_t)n * qg * N * sizeof(double));
    double *us = (double *)malloc((size_t)n * 3 * N * sizeof(double));
    double *lam = (double *)calloc((size_t)qg * N, sizeof(double));
    double *lam2 = (double *)calloc((size_t)qg * N, sizeof(double));
    if (!gs || !us || !lam || !lam2) { free(gs); free(us); free(lam); free(lam2); return 2; }

    double J0 = s->reacted_total;
    for (long t = 0; t < n; ++t) {
        memcpy(gs + (size_t)t * qg * N, s->gpost, (size_t)qg * N * sizeof(double));
        one_step(s);
        memcpy(us + (size_t)t * 3 * N, s->usol, (size_t)3 * N * sizeof(double));
    }
    *J = s->reacted_total - J0;
    double gk = 0.0, gc = 0.0;
    if (dJ_dkfield) memset(dJ_dkfield, 0, N * sizeof(double));

    for (long t = n - 1; t >= 0; --t) {
        const double *g = gs + (size_t)t * qg * N;
        const double *u = us + (size_t)t * 3 * N;
        memset(lam2, 0, (size_t)qg * N * sizeof(double));
        for (int z = 0; z < p->nz; ++z)
            for (int y = 0; y < p->ny; ++y)
                for (int x = 0; x < p->nx; ++x) {
                    long id = IDX(s, x, y, z);
                    if (s->cls[id] == ORC_SOLID) continue;
                    /* forward pull of this cell (kept to know h_obar) */
                    double hh[19];
                    int st[19];
                    long src[19];
                    double Cold = 0.0;
                    for (int i = 0; i < qg; ++i) Cold += g[i * N + id];
                    for (int i = 0; i < qg; ++i) {
                        int me[3] = {-G->e[i][0], -G->e[i][1], -G->e[i][2]};
                        st[i] = neighbour(s, x, y, z, me, &src[i]);
                        double bb = g[G->opp[i] * N + id];
                        if (st[i] == NB_IN && s->cls[src[i]] != ORC_SOLID) hh[i] = g[i * N + src[i]];
                        else if (st[i] == NB_INLET && s->cls[id] == ORC_FLUID) hh[i] = -bb + 2.0 * G->w[i] * p->c_inlet;
                        else if (st[i] == NB_OUTLET && s->cls[id] == ORC_FLUID) hh[i] = -bb + 2.0 * G->w[i] * Cold;
                        else hh[i] = bb;
                    }
                    /* collision transpose: a_h'[j] = sum_i lambda_i M[i][j] */
                    double uu[3] = {u[3 * id], u[3 * id + 1], u[3 * id + 2]};
                    double ah[19];
                    for (int j = 0; j < qg; ++j) {
                        double col[19], geq[19];
                        for (int i = 0; i < qg; ++i) col[i] = (i == j) ? 1.0 : 0.0;
                        solute_equilibrium(G, 1.0, uu, geq);
                        collide(G, col, geq, trt_g, tg_sym, tg_anti);
                        double a = 0.0;
                        for (int i = 0; i < qg; ++i) a += lam[i * N + id] * col[i];
                        ah[j] = a;
                    }
                    /* reactive boundary condition and ledger, transposed */
                    double ahh[19];
                    for (int i = 0; i < qg; ++i) ahh[i] = ah[i];
                    if (s->cls[id] == ORC_BOUND) {
                        int dir = s->kind[id] == ORC_KIND_DIRICHLET;
                        double kr = s->kfield ? s->kfield[id] : p->k_r;
                        double cell_k = 0.0;
                        for (int o = 1; o < qg; ++o) {
                            long nb;
                            if (neighbour(s, x, y, z, G->e[o], &nb) != NB_IN || s->cls[nb] != ORC_FLUID) continue;
                            int ob = G->opp[o];
                            /* h'_o replaced h_o: h_o reaches nothing but the ledger's -h_o */
                            double a = ah[o];
                            ahh[o] -= a;
                            if (dir) {           /* h'_o = -h_obar + 2 w C_dir, not in J */
                                ahh[ob] += -a;
                                continue;
                            }
                            a += 1.0;            /* the ledger's +h'_o */
                            ahh[o] += -1.0;      /* ... and its -h_o */
                            if (kr == 0.0) {     /* inert: h'_o = h_obar */
                                ahh[ob] += a;
                                continue;
                            }
                            double k, dkdkr;
                            int inf;
                            link_k(s, id, o, kr, &k, &dkdkr, &inf);
                            if (inf) {           /* h'_o = -h_obar + 2 w c_eq */
                                ahh[ob] += -a;
                                gc += a * 2.0 * G->w[o];
                                continue;
                            }
                            ahh[ob] += a * (1.0 - k) / (1.0 + k);
                            double dh = (2.0 * G->w[o] * p->c_eq - 2.0 * hh[ob]) / ((1.0 + k) * (1.0 + k));
                            cell_k += a * dh * dkdkr;
                            gc += a * k / (1.0 + k) * 2.0 * G->w[o];
                        }
                        gk += cell_k;
                        if (dJ_dkfield) dJ_dkfield[id] += cell_k;
                    }
                    /* pull transposed: scatter onto the previous state */
                    for (int i = 0; i < qg; ++i) {
                        int ib = G->opp[i];
                        if (st[i] == NB_IN && s->cls[src[i]] != ORC_SOLID) lam2[i * N + src[i]] += ahh[i];
                        else if (st[i] == NB_INLET && s->cls[id] == ORC_FLUID) lam2[ib * N + id] -= ahh[i];
                        else if (st[i] == NB_OUTLET && s->cls[id] == ORC_FLUID) {
                            lam2[ib * N + id] -= ahh[i];
                            for (int j = 0; j < qg; ++j) lam2[j * N + id] += 2.0 * G->w[i] * ahh[i];
                        } else lam2[ib * N + id] += ahh[i];
                    }
                }
        double *tmp = lam; lam = lam2; lam2 = tmp;
    }
    *dJ_dk = gk;
    *dJ_dceq = gc;
    free(gs); free(us); free(lam); free(lam2);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Building blocks exposed for the pins of the oracle itself.          */
/* ------------------------------------------------------------------ */
int orc_lattice(int q, int dim, double J0, int *e, double *w, double *cs2, int *opp)
{
    orc_lat L;
    if (make_lattice(&L, q, dim, J0)) return 1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    *cs2 = L.cs2;
    return 0;
}

int orc_equilibrium(int q, int dim, double J0, int solute, double dens, const double *u, double *out)
{
    orc_lat L;
    if (make_lattice(&L, q, dim, J0)) return 1;
    if (solute) solute_equilibrium(&L, dens, u, out);
    else flow_equilibrium(&L, dens, u, out);
    return 0;
}

double orc_rbc(double k, double w, double c_eq, double gt, int infinite)
{
    return rbc_value(k, w, c_eq, gt, infinite);
}
