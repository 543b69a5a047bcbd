/*
 * swe_oracle.c -- FP64 CPU oracle for the shallow-water finite-volume step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (Delmas & Soulaimani, "Multi-GPU implementation of a
 * time-explicit finite volume solver for the Shallow-Water Equations",
 * Sections 2-3):
 *   - conservative 2D shallow-water system U = (h, hu, hv)            (Eq 1-5)
 *   - cell-centred finite volumes on triangles, sum over the 3 edges  (Eq 6-11)
 *   - rotational invariance, Riemann problem in the edge normal frame (Eq 12-14)
 *   - boundary conditions: transmissive, inflow, wall                 (Sec 3.1)
 *   - explicit Euler in time, CFL on the inscribed radius             (Eq 15-16)
 *   - HLL flux with adaptive PVRS / TRRS / TSRS depth estimate        (Eq 17-23)
 *   - HLLC third component and dry-bed wave speeds                    (Eq 24-26)
 *   - hydrostatic reconstruction of the bed source                    (Eq 28-30)
 *   - semi-implicit Manning friction                                  (Eq 31-37)
 *
 * Readings of garbled or silent passages (all listed in the design notes):
 *   Eq 20  p_k = sqrt(h*(h*+h_k)/2)/h_k  (the printed "/2" is read as "/h_k")
 *   Eq 21  the velocity jump is the normal velocity un_R - un_L
 *   Eq 22  un_L - un_R; the base is clamped at 0 before squaring (vacuum)
 *   Eq 24  upwind: ut_L when S* >= 0, ut_R when S* < 0
 *   Eq 26  the second line is the right-dry case; "dry" means h <= h_dry;
 *          both sides dry gives a zero flux
 *   Eq 30  the bed source carries a factor 1/2: (g/2)(h**^2 - h^2) n
 *   Eq 37  the stray "|Omega_i|" / ".n_i" factors are dropped
 *   Sec 3.1 wall/inflow pressure term is g h^2/2; inflow is inward, so the
 *          outward-normal mass flux is -q with q = Q / (length of the group)
 *   fixed-stage boundary (not in the paper): ghost depth max(0, eta_s - z_i)
 *          with the cell's velocity, solved by the same Riemann flux
 *   after the update: h < 0 is clamped to 0 (with hu = hv = 0) and counted;
 *          a cell with h <= h_dry has its momentum set to zero
 *
 * The code is deliberately plain: one loop over cells, one loop over the
 * three edges of each cell, every edge flux evaluated from the cell's own
 * point of view (left state = this cell, normal = this cell's outward normal).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EMESH 2
#define ORC_ENOMEM 3

#define ORC_BC_WALL 0
#define ORC_BC_INFLOW 1
#define ORC_BC_TRANSMISSIVE 2
#define ORC_BC_STAGE 3

#define ORC_MAX_GROUPS 64

typedef struct {
    int64_t n_nodes, n_cells;
    double g, h_dry;
    const double *node_x, *node_y; /* views into a private copy */
    double *nodes;                 /* [n_nodes][2] copy */
    int32_t *tri;                  /* [n_cells][3], counter-clockwise copy */
    double *z, *m;                 /* [n_cells] bed elevation, Manning n */
    double *area, *rin;            /* [n_cells] area and inscribed radius */
    double *len, *nx, *ny;         /* [n_cells][3] edge length and outward unit normal */
    int64_t *nbr;                  /* [n_cells][3] neighbour cell, or -1 - group */
    /* boundary groups: group 0 is the default wall */
    int n_groups;
    int kind[ORC_MAX_GROUPS];
    double value[ORC_MAX_GROUPS];  /* Q (m^3/s) for inflow, eta_s (m) for stage */
    double glen[ORC_MAX_GROUPS];   /* total edge length of the group */
    int hll_only;                  /* 1: HLL for all three components (Eq 17-18) */
} orc_mesh;

/* ------------------------------------------------------------------------ */
/* Mesh: orientation, neighbours by shared edge, geometry                    */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t a, b, cell; int32_t j; } orc_edge_rec;

static int orc_edge_cmp(const void* p, const void* q) {
    const orc_edge_rec* e = (const orc_edge_rec*)p;
    const orc_edge_rec* f = (const orc_edge_rec*)q;
    if (e->a != f->a) return e->a < f->a ? -1 : 1;
    if (e->b != f->b) return e->b < f->b ? -1 : 1;
    if (e->cell != f->cell) return e->cell < f->cell ? -1 : 1;
    return e->j - f->j;
}

void orc_mesh_free(orc_mesh* M) {
    if (!M) return;
    free(M->nodes); free(M->tri); free(M->z); free(M->m);
    free(M->area); free(M->rin); free(M->len); free(M->nx); free(M->ny);
    free(M->nbr);
    free(M);
}

/* Builds the oracle's mesh: copies the inputs, orients every triangle
 * counter-clockwise, finds the cell across each edge (the neighbours of
 * Section 4.2: cells sharing an edge), and computes |Omega_i|, L_ij, the
 * outward unit normal n_ij (Eq 9) and the inscribed radius R = 2|Omega|/P
 * used by the CFL condition (Eq 15).  Every boundary edge starts as a wall. */
orc_mesh* orc_mesh_new(const double* nodes, int64_t n_nodes, const int32_t* tris,
                       int64_t n_cells, const double* z, const double* m,
                       double g, double h_dry, int* err) {
    *err = ORC_OK;
    if (n_nodes < 3 || n_cells < 1 || !nodes || !tris || !z || !m) { *err = ORC_EINVAL; return NULL; }
    orc_mesh* M = (orc_mesh*)calloc(1, sizeof(orc_mesh));
    if (!M) { *err = ORC_ENOMEM; return NULL; }
    M->n_nodes = n_nodes; M->n_cells = n_cells; M->g = g; M->h_dry = h_dry;
    M->nodes = (double*)malloc(sizeof(double) * 2 * n_nodes);
    M->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * n_cells);
    M->z = (double*)malloc(sizeof(double) * n_cells);
    M->m = (double*)malloc(sizeof(double) * n_cells);
    M->area = (double*)malloc(sizeof(double) * n_cells);
    M->rin = (double*)malloc(sizeof(double) * n_cells);
    M->len = (double*)malloc(sizeof(double) * 3 * n_cells);
    M->nx = (double*)malloc(sizeof(double) * 3 * n_cells);
    M->ny = (double*)malloc(sizeof(double) * 3 * n_cells);
    M->nbr = (int64_t*)malloc(sizeof(int64_t) * 3 * n_cells);
    orc_edge_rec* rec = (orc_edge_rec*)malloc(sizeof(orc_edge_rec) * 3 * n_cells);
    if (!M->nodes || !M->tri || !M->z || !M->m || !M->area || !M->rin || !M->len ||
        !M->nx || !M->ny || !M->nbr || !rec) {
        free(rec); orc_mesh_free(M); *err = ORC_ENOMEM; return NULL;
    }
    memcpy(M->nodes, nodes, sizeof(double) * 2 * n_nodes);
    memcpy(M->z, z, sizeof(double) * n_cells);
    memcpy(M->m, m, sizeof(double) * n_cells);

    for (int64_t i = 0; i < n_cells; ++i) {
        int32_t v0 = tris[3 * i], v1 = tris[3 * i + 1], v2 = tris[3 * i + 2];
        if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= n_nodes || v1 >= n_nodes || v2 >= n_nodes ||
            v0 == v1 || v1 == v2 || v0 == v2) {
            free(rec); orc_mesh_free(M); *err = ORC_EMESH; return NULL;
        }
        double x0 = nodes[2 * v0], y0 = nodes[2 * v0 + 1];
        double x1 = nodes[2 * v1], y1 = nodes[2 * v1 + 1];
        double x2 = nodes[2 * v2], y2 = nodes[2 * v2 + 1];
        double twice_area = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        if (twice_area == 0.0 || !isfinite(twice_area)) {
            free(rec); orc_mesh_free(M); *err = ORC_EMESH; return NULL;
        }
        if (twice_area < 0) { int32_t t = v1; v1 = v2; v2 = t; twice_area = -twice_area; }
        M->tri[3 * i] = v0; M->tri[3 * i + 1] = v1; M->tri[3 * i + 2] = v2;
        M->area[i] = 0.5 * twice_area;
        double perimeter = 0.0;
        for (int j = 0; j < 3; ++j) {
            int32_t a = M->tri[3 * i + j], b = M->tri[3 * i + (j + 1) % 3];
            double dx = nodes[2 * b] - nodes[2 * a];
            double dy = nodes[2 * b + 1] - nodes[2 * a + 1];
            double L = sqrt(dx * dx + dy * dy);
            /* counter-clockwise triangle: the interior lies to the left of the
               directed edge a->b, so the outward normal is (dy, -dx)/L */
            M->len[3 * i + j] = L;
            M->nx[3 * i + j] = dy / L;
            M->ny[3 * i + j] = -dx / L;
            perimeter += L;
            rec[3 * i + j].a = a < b ? a : b;
            rec[3 * i + j].b = a < b ? b : a;
            rec[3 * i + j].cell = i;
            rec[3 * i + j].j = j;
            M->nbr[3 * i + j] = -1; /* wall group 0 until a partner is found */
        }
        M->rin[i] = 2.0 * M->area[i] / perimeter;
    }
    qsort(rec, (size_t)(3 * n_cells), sizeof(orc_edge_rec), orc_edge_cmp);
    int64_t p = 0;
    while (p < 3 * n_cells) {
        int64_t q = p + 1;
        while (q < 3 * n_cells && rec[q].a == rec[p].a && rec[q].b == rec[p].b) ++q;
        int64_t cnt = q - p;
        if (cnt > 2) { free(rec); orc_mesh_free(M); *err = ORC_EMESH; return NULL; }
        if (cnt == 2) {
            if (rec[p].cell == rec[p + 1].cell) { free(rec); orc_mesh_free(M); *err = ORC_EMESH; return NULL; }
            M->nbr[3 * rec[p].cell + rec[p].j] = rec[p + 1].cell;
            M->nbr[3 * rec[p + 1].cell + rec[p + 1].j] = rec[p].cell;
        }
        p = q;
    }
    free(rec);
    M->n_groups = 1;
    M->kind[0] = ORC_BC_WALL;
    M->value[0] = 0.0;
    M->glen[0] = 0.0;
    for (int64_t s = 0; s < 3 * n_cells; ++s)
        if (M->nbr[s] < 0) M->glen[0] += M->len[s];
    return M;
}

/* Assigns the boundary edges listed as node pairs to a new boundary group
 * (Section 3.1).  Returns the group index, or a negative error. */
int orc_mesh_set_bc(orc_mesh* M, const int32_t* pairs, int64_t n, int kind, double value) {
    if (kind < ORC_BC_WALL || kind > ORC_BC_STAGE) return -ORC_EINVAL;
    if (M->n_groups >= ORC_MAX_GROUPS) return -ORC_EINVAL;
    int grp = M->n_groups;
    double total = 0.0;
    /* plain search: list the boundary edges once, then scan it for each pair */
    int64_t nb = 0;
    for (int64_t s = 0; s < 3 * M->n_cells; ++s) nb += M->nbr[s] < 0;
    int64_t* bslot = (int64_t*)malloc(sizeof(int64_t) * (nb > 0 ? nb : 1));
    if (!bslot) return -ORC_ENOMEM;
    nb = 0;
    for (int64_t s = 0; s < 3 * M->n_cells; ++s)
        if (M->nbr[s] < 0) bslot[nb++] = s;
    for (int64_t e = 0; e < n; ++e) {
        int32_t a = pairs[2 * e], b = pairs[2 * e + 1];
        int found = 0;
        for (int64_t r = 0; r < nb; ++r) {
            int64_t s = bslot[r], i = s / 3;
            int j = (int)(s % 3);
            int32_t u = M->tri[3 * i + j], v = M->tri[3 * i + (j + 1) % 3];
            if ((u == a && v == b) || (u == b && v == a)) {
                if (M->nbr[s] != -1 - grp) {
                    /* an edge moved out of an earlier group no longer counts there */
                    int old = (int)(-1 - M->nbr[s]);
                    M->glen[old] -= M->len[s];
                    total += M->len[s];
                }
                M->nbr[s] = -1 - grp;
                found = 1;
                break;
            }
        }
        if (!found) { free(bslot); return -ORC_EINVAL; }
    }
    free(bslot);
    M->kind[grp] = kind;
    M->value[grp] = value;
    M->glen[grp] = total;
    M->n_groups = grp + 1;
    return grp;
}

/* Copies the oracle's geometry out (for the preprocessing pins). */
void orc_mesh_geometry(const orc_mesh* M, double* area, double* rin, int64_t* nbr,
                       double* len, double* nx, double* ny) {
    int64_t n = M->n_cells;
    if (area) memcpy(area, M->area, sizeof(double) * n);
    if (rin) memcpy(rin, M->rin, sizeof(double) * n);
    if (nbr) memcpy(nbr, M->nbr, sizeof(int64_t) * 3 * n);
    if (len) memcpy(len, M->len, sizeof(double) * 3 * n);
    if (nx) memcpy(nx, M->nx, sizeof(double) * 3 * n);
    if (ny) memcpy(ny, M->ny, sizeof(double) * 3 * n);
}

int64_t orc_mesh_n_cells(const orc_mesh* M) { return M->n_cells; }

/* Boundary groups: kind, value (Q or eta_s) and total edge length of each;
 * returns the number of groups. */
int orc_mesh_groups(const orc_mesh* M, int* kind, double* value, double* glen) {
    for (int g = 0; g < M->n_groups; ++g) {
        if (kind) kind[g] = M->kind[g];
        if (value) value[g] = M->value[g];
        if (glen) glen[g] = M->glen[g];
    }
    return M->n_groups;
}

/* ------------------------------------------------------------------------ */
/* Riemann solver in the edge-normal frame (Eq 14, 17-26)                    */
/* ------------------------------------------------------------------------ */

/* Estimate of the star-region depth h*.  The first guess h0* (Eq 21) picks
 * the two-rarefaction estimate (Eq 22) or the two-shock estimate (Eq 23). */
double orc_hstar(double hL, double unL, double hR, double unR, double g, double* h0_out) {
    double aL = sqrt(g * hL), aR = sqrt(g * hR);
    double h0 = 0.5 * (hL + hR) - 0.25 * (unR - unL) * (hL + hR) / (aL + aR);
    if (h0_out) *h0_out = h0;
    double hmin = hL < hR ? hL : hR;
    if (h0 <= hmin) {
        double base = 0.5 * (aL + aR) + 0.25 * (unL - unR);
        if (base < 0.0) base = 0.0;
        return base * base / g;
    }
    double gL = sqrt(g * (h0 + hL) / (2.0 * h0 * hL));
    double gR = sqrt(g * (h0 + hR) / (2.0 * h0 * hR));
    return (hL * gL + hR * gR + unL - unR) / (gL + gR);
}

/* Physical flux in the normal direction, G(U) of Eq 1 with x -> n. */
static void orc_phys_flux(double h, double un, double ut, double g, double G[3]) {
    G[0] = h * un;
    G[1] = h * un * un + 0.5 * g * h * h;
    G[2] = h * un * ut;
}

/* HLLC flux G~(U_L, U_R) in the rotated frame, with U_K = (h_K, h_K un_K,
 * h_K ut_K).  speeds (optional) receives S_L, S_R, S*. */
void orc_hllc(double hL, double unL, double utL, double hR, double unR, double utR,
              double g, double h_dry, double G[3], double speeds[3]) {
    int dryL = hL <= h_dry, dryR = hR <= h_dry;
    if (dryL && dryR) {
        G[0] = G[1] = G[2] = 0.0;
        if (speeds) speeds[0] = speeds[1] = speeds[2] = 0.0;
        return;
    }
    double aL = sqrt(g * hL), aR = sqrt(g * hR);
    double SL, SR, Sstar;
    if (dryL) {                /* Eq 26, first line */
        SL = unR - 2.0 * aR;
        SR = unR + aR;
        Sstar = SL;
    } else if (dryR) {         /* Eq 26, second line (right side dry) */
        SL = unL - aL;
        SR = unL + 2.0 * aL;
        Sstar = SR;
    } else {
        double hs = orc_hstar(hL, unL, hR, unR, g, NULL);           /* Eq 21-23 */
        double pL = hs > hL ? sqrt(hs * (hs + hL) / 2.0) / hL : 1.0; /* Eq 20 */
        double pR = hs > hR ? sqrt(hs * (hs + hR) / 2.0) / hR : 1.0;
        SL = unL - aL * pL;                                          /* Eq 19 */
        SR = unR + aR * pR;
        Sstar = (SL * hR * (unR - SR) - SR * hL * (unL - SL)) /
                (hR * (unR - SR) - hL * (unL - SL));                 /* Eq 25 */
    }
    double GL[3], GR[3];
    orc_phys_flux(hL, unL, utL, g, GL);
    orc_phys_flux(hR, unR, utR, g, GR);
    if (SL >= 0.0) {                                                 /* Eq 17 */
        G[0] = GL[0]; G[1] = GL[1];
    } else if (SR <= 0.0) {
        G[0] = GR[0]; G[1] = GR[1];
    } else {                                                         /* Eq 18 */
        double UL[2] = {hL, hL * unL}, UR[2] = {hR, hR * unR};
        for (int c = 0; c < 2; ++c)
            G[c] = (SR * GL[c] - SL * GR[c] + SR * SL * (UR[c] - UL[c])) / (SR - SL);
    }
    G[2] = Sstar >= 0.0 ? G[0] * utL : G[0] * utR;                  /* Eq 24 */
    if (speeds) { speeds[0] = SL; speeds[1] = SR; speeds[2] = Sstar; }
}

/* HLL flux for all three components (Eq 17-18 applied to U_3 = h ut as
 * well), with the same wave-speed estimates as orc_hllc. */
void orc_hll(double hL, double unL, double utL, double hR, double unR, double utR,
             double g, double h_dry, double G[3]) {
    double S[3];
    orc_hllc(hL, unL, utL, hR, unR, utR, g, h_dry, G, S);
    if ((hL <= h_dry && hR <= h_dry)) return;          /* both dry: zero flux */
    double SL = S[0], SR = S[1];
    double GL3 = hL * unL * utL, GR3 = hR * unR * utR;
    if (SL >= 0.0) G[2] = GL3;
    else if (SR <= 0.0) G[2] = GR3;
    else G[2] = (SR * GL3 - SL * GR3 + SR * SL * (hR * utR - hL * utL)) / (SR - SL);
}

/* Selects the flux: 0 = HLLC (default), 1 = HLL. */
void orc_mesh_set_flux(orc_mesh* M, int hll_only) { M->hll_only = hll_only ? 1 : 0; }

/* ------------------------------------------------------------------------ */
/* Semi-implicit Manning friction (Eq 31-37)                                 */
/* ------------------------------------------------------------------------ */

/* Given the cell state U^n = (h, hu, hv) and the explicit right-hand side
 * R = (Rh, Rhu, Rhv) of Eq 37 (flux divergence plus bed source, per unit
 * area), returns dU = U^{n+1} - U^n solving
 *     [I - dt/2 J_f] dU = dt (R + S_f(U^n)).
 * S_f and its Jacobian J_f are written out entry by entry (Eq 32, 35) and the
 * 2x2 momentum block is solved by Cramer's rule. */
void orc_friction_update(double h, double hu, double hv, double Rh, double Rhu, double Rhv,
                         double m, double dt, double g, double h_dry, double dU[3]) {
    double dh = dt * Rh;
    if (!(h > h_dry) || !(m > 0.0)) {
        dU[0] = dh; dU[1] = dt * Rhu; dU[2] = dt * Rhv;
        return;
    }
    /* S_f = -g m^2 h^{-7/3} |q| q with q = (hu, hv) (Eq 32 in conservative form) */
    double c = g * m * m * pow(h, -7.0 / 3.0);
    double qn = sqrt(hu * hu + hv * hv);
    double Sx = -c * qn * hu, Sy = -c * qn * hv;
    /* J_f rows 2-3 (Eq 35): d/dh, d/dhu, d/dhv */
    double Jxh = (7.0 / 3.0) * c * qn * hu / h;
    double Jyh = (7.0 / 3.0) * c * qn * hv / h;
    double Jxx, Jxy, Jyx, Jyy;
    if (qn > 0.0) {
        Jxx = -c * (qn + hu * hu / qn);
        Jxy = -c * (hu * hv / qn);
        Jyx = -c * (hv * hu / qn);
        Jyy = -c * (qn + hv * hv / qn);
    } else {
        Jxx = 0.0; Jxy = 0.0; Jyx = 0.0; Jyy = 0.0;
    }
    /* [I - dt/2 J] dU = dt (R + S): row 1 gives dh; rows 2-3 give a 2x2 system */
    double A11 = 1.0 - 0.5 * dt * Jxx, A12 = -0.5 * dt * Jxy;
    double A21 = -0.5 * dt * Jyx, A22 = 1.0 - 0.5 * dt * Jyy;
    double b1 = dt * (Rhu + Sx) + 0.5 * dt * Jxh * dh;
    double b2 = dt * (Rhv + Sy) + 0.5 * dt * Jyh * dh;
    double det = A11 * A22 - A12 * A21;
    dU[0] = dh;
    dU[1] = (b1 * A22 - A12 * b2) / det;
    dU[2] = (A11 * b2 - b1 * A21) / det;
}

/* ------------------------------------------------------------------------ */
/* One explicit Euler step (Eq 16 / 27 / 37)                                  */
/* ------------------------------------------------------------------------ */

/* Right-hand side of cell i (per unit area): -1/|Omega| sum_j L_ij F_ij
 * plus the hydrostatic-reconstruction bed source (Eq 30). */
static void orc_cell_rhs(const orc_mesh* M, int64_t i, const double* h, const double* hu,
                         const double* hv, double R[3]) {
    const double g = M->g, h_dry = M->h_dry;
    double hi = h[i], zi = M->z[i];
    double ui = 0.0, vi = 0.0;
    if (hi > h_dry) { ui = hu[i] / hi; vi = hv[i] / hi; }
    double flux[3] = {0.0, 0.0, 0.0};
    double src[2] = {0.0, 0.0};
    for (int j = 0; j < 3; ++j) {
        double L = M->len[3 * i + j];
        double n1 = M->nx[3 * i + j], n2 = M->ny[3 * i + j];
        int64_t k = M->nbr[3 * i + j];
        double G[3];
        if (k >= 0) {
            double hk = h[k], zk = M->z[k];
            double uk = 0.0, vk = 0.0;
            if (hk > h_dry) { uk = hu[k] / hk; vk = hv[k] / hk; }
            double zs = zi > zk ? zi : zk;                       /* interface bed */
            double hLs = hi + zi - zs; if (hLs < 0.0) hLs = 0.0; /* h**_ij (Eq 28) */
            double hRs = hk + zk - zs; if (hRs < 0.0) hRs = 0.0; /* h**_ji */
            double unL = ui * n1 + vi * n2, utL = -ui * n2 + vi * n1;   /* T_n (Eq 12) */
            double unR = uk * n1 + vk * n2, utR = -uk * n2 + vk * n1;
            if (M->hll_only) orc_hll(hLs, unL, utL, hRs, unR, utR, g, h_dry, G);
            else orc_hllc(hLs, unL, utL, hRs, unR, utR, g, h_dry, G, NULL);
            double s = 0.5 * g * (hLs * hLs - hi * hi);          /* Eq 30 with 1/2 */
            src[0] += L * s * n1;
            src[1] += L * s * n2;
        } else {
            int grp = (int)(-1 - k);
            int kind = M->kind[grp];
            if (kind == ORC_BC_WALL) {
                G[0] = 0.0; G[1] = 0.5 * g * hi * hi; G[2] = 0.0;
            } else if (kind == ORC_BC_INFLOW) {
                double q = M->value[grp] / M->glen[grp];
                G[0] = -q;
                G[1] = 0.5 * g * hi * hi + (hi > h_dry ? q * q / hi : 0.0);
                G[2] = 0.0;
            } else {
                double unL = ui * n1 + vi * n2, utL = -ui * n2 + vi * n1;
                double hg = hi;
                if (kind == ORC_BC_STAGE) { hg = M->value[grp] - zi; if (hg < 0.0) hg = 0.0; }
                if (M->hll_only) orc_hll(hi, unL, utL, hg, unL, utL, g, h_dry, G);
                else orc_hllc(hi, unL, utL, hg, unL, utL, g, h_dry, G, NULL);
            }
        }
        /* back to (x, y): T_n^{-1} G (Eq 12) */
        double F0 = G[0];
        double F1 = G[1] * n1 - G[2] * n2;
        double F2 = G[1] * n2 + G[2] * n1;
        flux[0] += L * F0;
        flux[1] += L * F1;
        flux[2] += L * F2;
    }
    double A = M->area[i];
    R[0] = -flux[0] / A;
    R[1] = (-flux[1] + src[0]) / A;
    R[2] = (-flux[2] + src[1]) / A;
}

/* New state of cell i after one step of size dt. Returns 1 if h was clamped. */
static int orc_cell_update(const orc_mesh* M, int64_t i, const double* h, const double* hu,
                           const double* hv, double dt, double out[3]) {
    double R[3], dU[3];
    orc_cell_rhs(M, i, h, hu, hv, R);
    orc_friction_update(h[i], hu[i], hv[i], R[0], R[1], R[2], M->m[i], dt, M->g, M->h_dry, dU);
    out[0] = h[i] + dU[0];
    out[1] = hu[i] + dU[1];
    out[2] = hv[i] + dU[2];
    if (out[0] < 0.0) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return 1; }
    if (out[0] <= M->h_dry) { out[1] = 0.0; out[2] = 0.0; }
    return 0;
}

/* Threads of the OpenMP loops below, for timing the oracle on one core and
 * on all of them; results do not depend on it (each cell's update is a
 * separate computation, and the reductions are an integer sum and a min). */
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_max_threads(void) { return omp_get_max_threads(); }

/* One step for every cell.  Returns the number of clamped cells. */
int64_t orc_step(const orc_mesh* M, const double* h, const double* hu, const double* hv,
                 double dt, double* h_out, double* hu_out, double* hv_out) {
    int64_t clamped = 0;
#pragma omp parallel for schedule(static) reduction(+ : clamped)
    for (int64_t i = 0; i < M->n_cells; ++i) {
        double out[3];
        clamped += orc_cell_update(M, i, h, hu, hv, dt, out);
        h_out[i] = out[0]; hu_out[i] = out[1]; hv_out[i] = out[2];
    }
    return clamped;
}

/* One step for a list of cells only (sampled parity at large sizes). */
int64_t orc_step_cells(const orc_mesh* M, const double* h, const double* hu, const double* hv,
                       double dt, const int64_t* cells, int64_t n_sel,
                       double* h_out, double* hu_out, double* hv_out) {
    int64_t clamped = 0;
#pragma omp parallel for schedule(static) reduction(+ : clamped)
    for (int64_t s = 0; s < n_sel; ++s) {
        double out[3];
        clamped += orc_cell_update(M, cells[s], h, hu, hv, dt, out);
        h_out[s] = out[0]; hu_out[s] = out[1]; hv_out[s] = out[2];
    }
    return clamped;
}

/* Right-hand sides for every cell (pins on the flux divergence). */
void orc_rhs(const orc_mesh* M, const double* h, const double* hu, const double* hv,
             double* Rh, double* Rhu, double* Rhv) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M->n_cells; ++i) {
        double R[3];
        orc_cell_rhs(M, i, h, hu, hv, R);
        Rh[i] = R[0]; Rhu[i] = R[1]; Rhv[i] = R[2];
    }
}

/* CFL time step (Eq 15 with d = inscribed radius):
 * dt = cfl * min over wet cells of R_i / (sqrt(g h_i) + |u_i|).
 * Returns +inf when no cell is wet. */
double orc_dt(const orc_mesh* M, const double* h, const double* hu, const double* hv, double cfl) {
    double best = INFINITY;
#pragma omp parallel for schedule(static) reduction(min : best)
    for (int64_t i = 0; i < M->n_cells; ++i) {
        if (h[i] > M->h_dry) {
            double u = hu[i] / h[i], v = hv[i] / h[i];
            double c = M->rin[i] / (sqrt(M->g * h[i]) + sqrt(u * u + v * v));
            if (c < best) best = c;
        }
    }
    return cfl * best;
}

/* Outward discharge through each boundary group for the state (h, hu, hv):
 * Q_g = sum over the group's edges of L * (mass flux of Section 3.1's boundary
 * treatment), i.e. the mass leaving through those edges in the next step per
 * unit time.  Returns the number of groups written to Q. */
int orc_boundary_discharge(const orc_mesh* M, const double* h, const double* hu, const double* hv, double* Q) {
    const double g = M->g, h_dry = M->h_dry;
    for (int k = 0; k < M->n_groups; ++k) Q[k] = 0.0;
    for (int64_t i = 0; i < M->n_cells; ++i) {
        for (int j = 0; j < 3; ++j) {
            int64_t k = M->nbr[3 * i + j];
            if (k >= 0) continue;
            int grp = (int)(-1 - k);
            int kind = M->kind[grp];
            double hi = h[i], ui = 0.0, vi = 0.0;
            if (hi > h_dry) { ui = hu[i] / hi; vi = hv[i] / hi; }
            double n1 = M->nx[3 * i + j], n2 = M->ny[3 * i + j];
            double G0;
            if (kind == ORC_BC_WALL) {
                G0 = 0.0;
            } else if (kind == ORC_BC_INFLOW) {
                G0 = -M->value[grp] / M->glen[grp];
            } else {
                double un = ui * n1 + vi * n2, ut = -ui * n2 + vi * n1;
                double hg = hi;
                if (kind == ORC_BC_STAGE) { hg = M->value[grp] - M->z[i]; if (hg < 0.0) hg = 0.0; }
                double G[3];
                orc_hllc(hi, un, ut, hg, un, ut, g, h_dry, G, NULL);
                G0 = G[0];
            }
            Q[grp] += M->len[3 * i + j] * G0;
        }
    }
    return M->n_groups;
}

/* nsteps steps in place, the time step recomputed after every update.
 * t is advanced by the sum of the steps.  Returns the number of clamps, or
 * -1 if every cell is dry (no time step exists). */
int64_t orc_run(const orc_mesh* M, double* h, double* hu, double* hv, int64_t nsteps,
                double cfl, double* t, double* dt_log) {
    int64_t n = M->n_cells, clamped = 0;
    double* h2 = (double*)malloc(sizeof(double) * n);
    double* hu2 = (double*)malloc(sizeof(double) * n);
    double* hv2 = (double*)malloc(sizeof(double) * n);
    if (!h2 || !hu2 || !hv2) { free(h2); free(hu2); free(hv2); return -2; }
    for (int64_t s = 0; s < nsteps; ++s) {
        double dt = orc_dt(M, h, hu, hv, cfl);
        if (!isfinite(dt)) { clamped = -1; break; }
        if (dt_log) dt_log[s] = dt;
        clamped += orc_step(M, h, hu, hv, dt, h2, hu2, hv2);
        memcpy(h, h2, sizeof(double) * n);
        memcpy(hu, hu2, sizeof(double) * n);
        memcpy(hv, hv2, sizeof(double) * n);
        if (t) *t += dt;
    }
    free(h2); free(hu2); free(hv2);
    return clamped;
}

/* nsteps steps with a prescribed time-step sequence (for gradient checks
 * that freeze dt at the values of a reference run). */
int64_t orc_run_fixed_dt(const orc_mesh* M, double* h, double* hu, double* hv, int64_t nsteps,
                         const double* dts) {
    int64_t n = M->n_cells, clamped = 0;
    double* h2 = (double*)malloc(sizeof(double) * n);
    double* hu2 = (double*)malloc(sizeof(double) * n);
    double* hv2 = (double*)malloc(sizeof(double) * n);
    if (!h2 || !hu2 || !hv2) { free(h2); free(hu2); free(hv2); return -2; }
    for (int64_t s = 0; s < nsteps; ++s) {
        clamped += orc_step(M, h, hu, hv, dts[s], h2, hu2, hv2);
        memcpy(h, h2, sizeof(double) * n);
        memcpy(hu, hu2, sizeof(double) * n);
        memcpy(hv, hv2, sizeof(double) * n);
    }
    free(h2); free(hu2); free(hv2);
    return clamped;
}

/* Replaces the bed elevation and Manning coefficients (gradient checks). */
void orc_mesh_set_fields(orc_mesh* M, const double* z, const double* m) {
    if (z) memcpy(M->z, z, sizeof(double) * M->n_cells);
    if (m) memcpy(M->m, m, sizeof(double) * M->n_cells);
}
