/*
 * FastQSL oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the method of Zhang, Chen, Liu & Wang
 * (2022), "FastQSL: A Fast Computation Method for Quasi-separatrix Layers"
 * (ApJL, arXiv:2208.12569). Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file; the product library never
 * does, and the two share no code, header, table or helper.
 *
 * What it computes, in the paper's order:
 *   - the field-line equation dr/ds = B/|B| (Sec. 2.1, Eq. rb), integrated with
 *     Fehlberg's RKF45 (Sec. 2.3) with the error measured in grid cells;
 *   - B between nodes by trilinear interpolation with a floor cell lookup
 *     (Sec. 2.2, Eqs. interp, w0, w1);
 *   - the twist number Tw = int (curl B . B)/(4 pi B^2) dl (Sec. 1, Eq. tw) from
 *     a curl grid, and the field-line length (Sec. 2.4);
 *   - the squashing factor Q by Method I (neighbour footpoint differences on an
 *     auxiliary plane S0, Sec. 2.1 Eqs. D+-2, D+-3, Q+-, Bn1; per-line tolerance
 *     and local rotation of S0, Sec. 4 Eqs. step/tol) and by Method II
 *     (deviation vectors, Sec. 2.1 Eqs. rb2, q_scott; gradient of B/B by the
 *     node grid of Eq. grad_B or by +-0.001-cell differences, Sec. 4).
 *
 * Readings of points the paper leaves open (each is also used by the tests):
 *   R1  Integration runs in index coordinates xi = (r - origin)/spacing with
 *       d xi/d tau = bt/|bt|, bt_a = B_a/spacing_a, so tau, step and tol are in
 *       cells (Sec. 2.3: "the unit of tol is the original grid spacing"). The
 *       physical length obeys dl/dtau = |B|/|bt| and dTw/dtau = (J.B)/(4 pi B^2)
 *       dl/dtau; length and Tw are two extra ODE components.
 *   R2  RKF45 = Fehlberg's 4(5) pair; the 4th-order solution is propagated; err =
 *       Euclidean norm of the position difference of the two solutions (cells).
 *       Accept if err <= tol. With q = (tol/err)^(1/4), computed as
 *       sqrt(sqrt(tol/err)): accept: h *= min(4, 0.9 q) (x4 if err = 0);
 *       reject: h *= max(0.1, 0.9 q). h stays in [h_min, h_max]; a reject at
 *       h_min is accepted and flagged STALL. Every trial (and every exit
 *       attempt) counts toward max_steps over both directions of a line. The
 *       paper does not give the controller; the fourth root is taken with the
 *       correctly rounded square root because the adaptive step sequence
 *       amplifies a one-ulp difference in h by orders of magnitude per step, so
 *       a pow() that differs between math libraries would make the sequence
 *       unreproducible.
 *   R3  Interpolation clamps the cell index to [0, n-2]; outside the box this is
 *       linear extrapolation from the boundary cell.
 *   R4  Curl and the B/B gradient use 2nd-order central differences inside and
 *       2nd-order one-sided differences on the faces (first order if n = 2).
 *   R5  Exit ("move one step back", Sec. 2.1): an accepted step whose end lies
 *       outside the closed box is discarded; the exit face is the face whose
 *       plane the chord prev->new crosses first (ties: lower axis first). From
 *       the previous point one RKF45 step (4th order, no error control) is taken
 *       with the face-normal index coordinate as independent variable (Henon
 *       1982), landing exactly on the face. If the result is outside on another
 *       axis, the step is redone toward that axis' face (3 faces at most, then
 *       the point is clamped into the box). If the face-normal velocity at any
 *       stage is below 1e-3 or points inward (grazing), h is halved and a normal
 *       step retaken; once h/2 < h_min the footpoint is the chord's crossing
 *       point (flag CHORD).
 *   R6  A direction whose first step exits through the seed's own face has
 *       length 0 (its footpoint is the seed).
 *   R12 End order: end 1 (S1) is the footpoint on the -n0 side of S0, traced
 *       first along -sign(B.n0) B; end 2 (S2) the other. On a box-face plane
 *       end 1 is therefore always the seed itself, and across a polarity
 *       inversion line the neighbours' ends stay matched (ordering ends by
 *       trace direction would mix seeds and far footpoints in the differences
 *       of R8). Lattice lines (also under Method II) are ordered by the
 *       lattice's n0; the four extra lines of a rotated S0 by sign(B0.n0) B0/|B0|
 *       so that they match their centre line; lines without an S0 (twist lists)
 *       have the backward end as end 1.
 *   R7  Seeds of a lattice are cell-centred: r(i,j,k) = o + (i+1/2) a1 +
 *       (j+1/2) a2 + (k+1/2) a3 (a3 = 0 for a plane); S0 is the plane spanned
 *       by a1, a2; the refined spacing delta of Sec. 2.1 is |a1| (resp. |a2|).
 *   R8  Method I: J_e = d(face coords of end e)/d(S0 coords), face coords being
 *       the two non-normal physical coordinates in increasing axis order. Per end
 *       and lattice axis: central difference if both neighbours end on the
 *       centre's face, one-sided if exactly one does, otherwise Q = NaN and
 *       status MIXED (Code2016 gave NaN, Sec. 2.1). Then
 *       Q = |J2 adj(J1)|_F^2 |Bn1 Bn2| / Bn0^2, which is Eqs. D+-2, D+-3, Q+-
 *       with det D replaced by |Bn1/Bn2| (Eq. Bn1).
 *   R9  Per-line tolerance (Sec. 4, Eq. tol): tol_line = tol_perp
 *       max(|Bn0/B|, rot_thresh)^1.5 (the power 1.5 as x sqrt(x), for the
 *       reason given in R2; other exponents use pow). On an interior S0 with |Bn0/B| <
 *       rot_thresh, S0 is rotated perpendicular to B (n0 = B/|B|, u = unit(b x
 *       e_m) for the axis m of smallest |b_m|, v = b x u), four extra lines
 *       are traced at r0 +- delta u, r0 +- delta v (delta = min(|a1|,|a2|)), all
 *       with tol_perp, and Bn0 = |B|. No rotation on a box face (the extra
 *       seeds would start outside); there the max() keeps the tolerance finite.
 *   R10 Method II: S0 is always perpendicular to B (Sec. 4), U0, V0 = the u, v
 *       of R9, tol = tol as given; dU/ds = (U . grad)(B/B), integrated in physical
 *       coordinates alongside R1; Q by Eq. q_scott with absolute values.
 *   R17 Q_perp (Sec. 2.1, after Titov 2007): S1 and S2 turned perpendicular to
 *       the line at its ends, so in Eq. q_scott n = B/|B| at each end: U~ = U -
 *       (U . B)/(B . B) B and B_n,e = |B_e|; with S0 perpendicular to B as in
 *       R10, Q_perp = |U~1^2 V~2^2 + U~2^2 V~1^2 - 2 (U~1.V~1)(U~2.V~2)|
 *       |B1| |B2| / |B0|^2. Method II only (the paper notes Method I's
 *       difficulty with it).
 *   R11 Line status bits: MAXSTEPS 1, NULL_B 2 (|bt| = 0 or not finite at an
 *       evaluation), STALL 4, MIXED 8, OUTSIDE 16 (seed outside the box),
 *       ROTATED 32, CHORD 64. Q and Tw are NaN when MAXSTEPS, NULL_B or OUTSIDE
 *       is set; Q is NaN when MIXED is set. MIXED describes the stencil of a
 *       good line's Q, so a line with MAXSTEPS, NULL_B or OUTSIDE never has it.
 *   R16 Stretched (rectilinear) grids, Sec. 2.2 and 2.3: the nodes are
 *       x_i, y_j, z_k from three increasing coordinate arrays. The cell of a
 *       point is the largest i in [0, n-2] with x_i <= x (a binary search;
 *       points below x_0 and NaN map to cell 0), and the weights are Eqs. w0,
 *       w1 as written, omega_0 = (x_{i+1} - x)/(x_{i+1} - x_i). The state is the
 *       physical position. Each trial step takes the widths D_a of the cell
 *       holding its start point and integrates dr/dtau = B/|bt| with bt_a =
 *       B_a/D_a: the step is step x scaling and the tolerance tol x scaling of
 *       the paper's stretched-grid rule, with scaling = |B|/|bt| evaluated
 *       along the step instead of once per cell. The error is |(r5 - r4)_a/D_a|
 *       (cells of the start cell), so on a uniform grid this is R1-R2 in exact
 *       arithmetic. The exit step uses x_a itself as the independent variable;
 *       its grazing test is on (dr_a/dtau)/D_a. Curl B uses the 2nd-order
 *       three-point differences of a non-uniform axis (the derivative of the
 *       quadratic through the three nodes; one-sided on the faces), which are
 *       the R4 stencils on a uniform axis. Method II: the grad(B/B) grid of
 *       way 1 takes the same three-point differences; way 2 offsets +-eps2
 *       cells of the step's start cell (eps2 D_a) and divides by 2 eps2 D_a.
 *   R18 Fixed-step scheme (Sec. 2.3, Kutta's 3/8-rule RK4; Sec. 4 Eq. step):
 *       with scheme = 1 every trial is one 3/8-rule step of the line's fixed size
 *       (cells, index space as in R1; length and Tw ride along) and is always
 *       accepted. A Method I lattice seed steps max(step_perp |Bn0/B|,
 *       step_min) (Eq. step); rotated seeds and their extra lines, Method II
 *       lines and seed lists step step_perp (the perpendicular case). The exit
 *       is R5 with 3/8-rule stages; a grazing exit halves the step, which then
 *       stays halved, down to h_min before the chord fallback. The paper gives
 *       no step_min; the library's default is step_perp x rot_thresh (the
 *       obliquity floor of R9). On a stretched grid (R16) the step is in cells
 *       of each trial's start cell.
 *   R13 Derivatives (the paper has none; the adjoint tests): d(Q, Tw)/dB is
 *       that of the traced computation with each line's accepted step sizes,
 *       exit faces and exit kinds (exit step, clamped exit step, chord after
 *       an exiting step of size h) frozen; rejected trials then contribute
 *       nothing. Everything else -- the curl grid, stage positions, the exit
 *       step's length to the face, the chord parameter, Bn at the seed and at
 *       both ends, the finite-difference stencils' values -- varies with B.
 *       oracle_lattice_log exports the frozen sequence; oracle/adjoint.py
 *       replays and differentiates it. With the fixed-step scheme (R18) the
 *       frozen sequence is the line's fixed steps (halved where an exit grazed).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846
#define NSTATE 11 /* xi(3), length, Tw, U(3), V(3) */

enum {
    ST_MAXSTEPS = 1,
    ST_NULL = 2,
    ST_STALL = 4,
    ST_MIXED = 8,
    ST_OUTSIDE = 16,
    ST_ROTATED = 32,
    ST_CHORD = 64
};
#define ST_BAD (ST_MAXSTEPS | ST_NULL | ST_OUTSIDE)

typedef struct {
    int method;          /* 1 = neighbour differences, 2 = deviation vectors */
    int way;             /* Method II gradient of B/B: 1 node grid, 2 +-eps */
    double tol;          /* tol_perp (Method I) / tol (Method II, twist), cells */
    double h0, hmin, hmax;
    long long max_steps;
    double rot_thresh;   /* 0.05 */
    double tol_exp;      /* 1.5 */
    double graze;        /* 1e-3 */
    double eps2;         /* 1e-3 cells */
    int qperp;           /* Method II: 1 = Q_perp (R17) */
    int scheme;          /* 0 = RKF45 (R2), 1 = fixed-step 3/8-rule RK4 (R18) */
    double step;         /* R18: step_perp (cells) */
    double step_min;     /* R18: lower bound of Eq. step (cells) */
} OParams;

typedef struct {
    long long n[3];
    double o[3], d[3];
    const double *B, *J, *G;
    const double *X[3]; /* stretched grid (R16): node coordinates per axis; NULL = uniform */
} OField;

typedef struct {
    double end[2][NSTATE]; /* [0] = backward end (S1), [1] = forward end (S2) */
    double Bend[2][3];
    int face[2];
    long long steps;
    int status;
} OLine;

/* Optional record of the accepted steps of a line (for the adjoint tests):
 * code 99 starts a direction (h = its sign), 0 is an accepted step of size h,
 * 16 + face the exit step onto that face, 40 + face the same when the point
 * had to be clamped into the box, 48 + face a chord fallback after an exiting
 * step of size h. */
typedef struct {
    double *h;
    int *code;
    int cap, n, overflow;
} OLog;

static void o_log(OLog *g, double h, int code)
{
    if (!g) return;
    if (g->n >= g->cap) {
        g->overflow = 1;
        return;
    }
    g->h[g->n] = h;
    g->code[g->n] = code;
    g->n++;
}

/* ------------------------------------------------------------------ */
/* node differences (R4) and the curl / B-hat gradient grids           */

static double o_dnode(const double *f, int nc, int c, long long node, long long stride,
                      long long i, long long n, double h)
{
#define F_(k) f[(node + ((long long)(k) - i) * stride) * nc + c]
    if (n == 2) return (F_(1) - F_(0)) / h;
    if (i == 0) return (-3.0 * F_(0) + 4.0 * F_(1) - F_(2)) / (2.0 * h);
    if (i == n - 1) return (3.0 * F_(n - 1) - 4.0 * F_(n - 2) + F_(n - 3)) / (2.0 * h);
    return (F_(i + 1) - F_(i - 1)) / (2.0 * h);
#undef F_
}

/* d f/d x_a at node index i along an axis with node coordinates X (R16):
 * the derivative of the quadratic through three neighbouring nodes,
 * one-sided at the ends, first order when n = 2. */
static double o_dnode_rect(const double *f, int nc, int c, long long node, long long stride, long long i,
                           long long n, const double *X)
{
#define F_(k) f[(node + ((long long)(k) - i) * stride) * nc + c]
    if (n == 2) return (F_(1) - F_(0)) / (X[1] - X[0]);
    if (i == 0) {
        double h1 = X[1] - X[0], h2 = X[2] - X[1];
        return -(2.0 * h1 + h2) / (h1 * (h1 + h2)) * F_(0) + (h1 + h2) / (h1 * h2) * F_(1) -
               h1 / (h2 * (h1 + h2)) * F_(2);
    }
    if (i == n - 1) {
        double h1 = X[n - 2] - X[n - 3], h2 = X[n - 1] - X[n - 2];
        return h2 / (h1 * (h1 + h2)) * F_(n - 3) - (h1 + h2) / (h1 * h2) * F_(n - 2) +
               (h1 + 2.0 * h2) / (h2 * (h1 + h2)) * F_(n - 1);
    }
    double h1 = X[i] - X[i - 1], h2 = X[i + 1] - X[i];
    return -h2 / (h1 * (h1 + h2)) * F_(i - 1) + (h2 - h1) / (h1 * h2) * F_(i) + h1 / (h2 * (h1 + h2)) * F_(i + 1);
#undef F_
}

/* J = curl B at every node of a stretched grid; X = x (n0), y (n1), z (n2)
 * coordinates back to back. */
int oracle_curl_rect(const double *B, const long long n[3], const double *X, double *J)
{
    if (n[0] < 2 || n[1] < 2 || n[2] < 2) return 1;
    const double *xs = X, *ys = X + n[0], *zs = X + n[0] + n[1];
    long long sx = 1, sy = n[0], sz = n[0] * n[1];
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n[2]; k++)
        for (long long j = 0; j < n[1]; j++)
            for (long long i = 0; i < n[0]; i++) {
                long long node = (k * n[1] + j) * n[0] + i;
                double dyBz = o_dnode_rect(B, 3, 2, node, sy, j, n[1], ys);
                double dzBy = o_dnode_rect(B, 3, 1, node, sz, k, n[2], zs);
                double dzBx = o_dnode_rect(B, 3, 0, node, sz, k, n[2], zs);
                double dxBz = o_dnode_rect(B, 3, 2, node, sx, i, n[0], xs);
                double dxBy = o_dnode_rect(B, 3, 1, node, sx, i, n[0], xs);
                double dyBx = o_dnode_rect(B, 3, 0, node, sy, j, n[1], ys);
                J[node * 3 + 0] = dyBz - dzBy;
                J[node * 3 + 1] = dzBx - dxBz;
                J[node * 3 + 2] = dxBy - dyBx;
            }
    return 0;
}

/* G[a*3+b] = d(B_b/|B|)/dx_a at every node of a stretched grid (R16, the
 * stencils of oracle_curl_rect); X as there. */
int oracle_gradb_rect(const double *B, const long long n[3], const double *X, double *G)
{
    if (n[0] < 2 || n[1] < 2 || n[2] < 2) return 1;
    long long nn = n[0] * n[1] * n[2];
    double *bh = (double *)malloc((size_t)nn * 3 * sizeof(double));
    if (!bh) return 2;
    for (long long q = 0; q < nn; q++) {
        double m = sqrt(B[3 * q] * B[3 * q] + B[3 * q + 1] * B[3 * q + 1] + B[3 * q + 2] * B[3 * q + 2]);
        for (int c = 0; c < 3; c++) bh[3 * q + c] = m > 0 ? B[3 * q + c] / m : 0.0;
    }
    const double *Xa[3] = {X, X + n[0], X + n[0] + n[1]};
    long long stride[3] = {1, n[0], n[0] * n[1]};
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n[2]; k++)
        for (long long j = 0; j < n[1]; j++)
            for (long long i = 0; i < n[0]; i++) {
                long long node = (k * n[1] + j) * n[0] + i;
                long long idx[3] = {i, j, k};
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        G[node * 9 + a * 3 + b] = o_dnode_rect(bh, 3, b, node, stride[a], idx[a], n[a], Xa[a]);
            }
    free(bh);
    return 0;
}

/* J = curl B at every node (the curl grid used by Eq. tw). */
int oracle_curl(const double *B, const long long n[3], const double d[3], double *J)
{
    if (n[0] < 2 || n[1] < 2 || n[2] < 2) return 1;
    long long sx = 1, sy = n[0], sz = n[0] * n[1];
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n[2]; k++)
        for (long long j = 0; j < n[1]; j++)
            for (long long i = 0; i < n[0]; i++) {
                long long node = (k * n[1] + j) * n[0] + i;
                double dyBz = o_dnode(B, 3, 2, node, sy, j, n[1], d[1]);
                double dzBy = o_dnode(B, 3, 1, node, sz, k, n[2], d[2]);
                double dzBx = o_dnode(B, 3, 0, node, sz, k, n[2], d[2]);
                double dxBz = o_dnode(B, 3, 2, node, sx, i, n[0], d[0]);
                double dxBy = o_dnode(B, 3, 1, node, sx, i, n[0], d[0]);
                double dyBx = o_dnode(B, 3, 0, node, sy, j, n[1], d[1]);
                J[node * 3 + 0] = dyBz - dzBy;
                J[node * 3 + 1] = dzBx - dxBz;
                J[node * 3 + 2] = dxBy - dyBx;
            }
    return 0;
}

/* G[a*3+b] = d(B_b/|B|)/dx_a at every node (Eq. grad_B; one-sided on faces).
 * A node with |B| = 0 contributes B/|B| = 0. */
int oracle_gradb(const double *B, const long long n[3], const double d[3], double *G)
{
    if (n[0] < 2 || n[1] < 2 || n[2] < 2) return 1;
    long long nn = n[0] * n[1] * n[2];
    double *bh = (double *)malloc((size_t)nn * 3 * sizeof(double));
    if (!bh) return 2;
    for (long long q = 0; q < nn; q++) {
        double m = sqrt(B[3 * q] * B[3 * q] + B[3 * q + 1] * B[3 * q + 1] + B[3 * q + 2] * B[3 * q + 2]);
        for (int c = 0; c < 3; c++) bh[3 * q + c] = m > 0 ? B[3 * q + c] / m : 0.0;
    }
    long long stride[3] = {1, n[0], n[0] * n[1]};
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < n[2]; k++)
        for (long long j = 0; j < n[1]; j++)
            for (long long i = 0; i < n[0]; i++) {
                long long node = (k * n[1] + j) * n[0] + i;
                long long idx[3] = {i, j, k};
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++)
                        G[node * 9 + a * 3 + b] = o_dnode(bh, 3, b, node, stride[a], idx[a], n[a], d[a]);
            }
    free(bh);
    return 0;
}

/* ------------------------------------------------------------------ */
/* trilinear interpolation (Sec. 2.2, Eqs. interp, w0, w1; R3)         */

/* stretched grid (R16): the cell of coordinate x on an axis with n nodes X */
static long long o_cell_rect(const double *X, long long n, double x)
{
    if (!(x >= X[0])) return 0; /* also NaN */
    long long lo = 0, hi = n - 2;  /* invariant: X[lo] <= x */
    while (lo < hi) {
        long long mid = (lo + hi + 1) / 2;
        if (X[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

static void o_interp(const OField *f, const double *arr, int nc, const double xi[3], double *out)
{
    long long i[3];
    double w[3][2];
    for (int a = 0; a < 3; a++) {
        if (f->X[a]) {
            /* stretched grid: binary search, Eq. w0 in physical coordinates */
            const double *X = f->X[a];
            i[a] = o_cell_rect(X, f->n[a], xi[a]);
            w[a][0] = (X[i[a] + 1] - xi[a]) / (X[i[a] + 1] - X[i[a]]);
            w[a][1] = 1.0 - w[a][0];
            continue;
        }
        double c = floor(xi[a]);            /* uniform grid: floor of x/spacing */
        if (!(c >= 0.0)) c = 0.0;           /* also maps NaN to cell 0 */
        if (c > (double)(f->n[a] - 2)) c = (double)(f->n[a] - 2);
        i[a] = (long long)c;
        w[a][0] = (c + 1.0) - xi[a];        /* (x_{i+1} - x)/(x_{i+1} - x_i), cells */
        w[a][1] = 1.0 - w[a][0];
    }
    for (int c = 0; c < nc; c++) out[c] = 0.0;
    for (int m = 0; m < 2; m++)
        for (int q = 0; q < 2; q++)
            for (int p = 0; p < 2; p++) {
                double wt = w[0][m] * w[1][q] * w[2][p];
                long long node = ((i[2] + p) * f->n[1] + (i[1] + q)) * f->n[0] + (i[0] + m);
                for (int c = 0; c < nc; c++) out[c] += wt * arr[node * nc + c];
            }
}

int oracle_interp(const double *arr, int nc, const long long n[3], const double *xi, long long np,
                  double *out)
{
    OField f;
    memset(&f, 0, sizeof f);
    for (int a = 0; a < 3; a++) f.n[a] = n[a];
    for (long long k = 0; k < np; k++) o_interp(&f, arr, nc, xi + 3 * k, out + (long long)nc * k);
    return 0;
}

/* ------------------------------------------------------------------ */
/* right-hand side of the field-line ODE (Eq. rb / Eq. rb2 in index space, R1) */

static int o_unit_b(const OField *f, const double xi[3], double bh[3])
{
    double B[3];
    o_interp(f, f->B, 3, xi, B);
    double m = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    if (!(m > 0) || !isfinite(m)) return 1;
    for (int c = 0; c < 3; c++) bh[c] = B[c] / m;
    return 0;
}

/* dy/dtau for the state y (ns = 5 or 11 comps); sigma = +1 forward, -1 backward;
 * D = the cell widths that normalise bt (the spacing on a uniform grid).
 * Returns 1 on a null / non-finite field. */
static int o_rhs(const OField *f, const OParams *p, const double *D, double sigma, int ns, const double *y,
                 double *dy)
{
    double B[3], bt[3];
    o_interp(f, f->B, 3, y, B);
    double bb = 0.0, BB = 0.0;
    for (int a = 0; a < 3; a++) {
        bt[a] = B[a] / D[a];
        bb += bt[a] * bt[a];
        BB += B[a] * B[a];
    }
    if (!(bb > 0.0) || !isfinite(bb)) return 1;
    double nbt = sqrt(bb), nB = sqrt(BB);
    if (f->X[0]) {
        /* stretched grid (R16): physical velocity B/|bt| */
        for (int a = 0; a < 3; a++) dy[a] = sigma * B[a] / nbt;
    } else {
        for (int a = 0; a < 3; a++) dy[a] = sigma * bt[a] / nbt;
    }
    double dl = nB / nbt; /* ds/dtau: physical arc length per cell of tau */
    dy[3] = dl;
    if (f->J) {
        double J[3];
        o_interp(f, f->J, 3, y, J);
        dy[4] = (J[0] * B[0] + J[1] * B[1] + J[2] * B[2]) / (4.0 * O_PI * BB) * dl; /* Eq. tw */
    } else {
        dy[4] = 0.0;
    }
    if (ns > 5) {
        /* grad(B/B): Gm[a][b] = d bhat_b / d x_a (physical) */
        double Gm[3][3];
        if (p->way == 1) {
            double g[9];
            o_interp(f, f->G, 9, y, g);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) Gm[a][b] = g[a * 3 + b];
        } else {
            for (int a = 0; a < 3; a++) {
                double xp[3] = {y[0], y[1], y[2]}, xm[3] = {y[0], y[1], y[2]};
                /* +-eps2 cells: of the grid (uniform; index state) or of the
                   step's start cell (stretched; physical state, R16) */
                double off = f->X[0] ? p->eps2 * D[a] : p->eps2, span = 2.0 * p->eps2 * D[a];
                xp[a] += off;
                xm[a] -= off;
                double bp[3], bm[3];
                if (o_unit_b(f, xp, bp) || o_unit_b(f, xm, bm)) return 1;
                for (int b = 0; b < 3; b++) Gm[a][b] = (bp[b] - bm[b]) / span;
            }
        }
        /* Eq. rb2: dU/ds = (U . grad)(B/B); ds = sigma * dl * dtau */
        for (int b = 0; b < 3; b++) {
            double su = 0.0, sv = 0.0;
            for (int a = 0; a < 3; a++) {
                su += y[5 + a] * Gm[a][b];
                sv += y[8 + a] * Gm[a][b];
            }
            dy[5 + b] = sigma * dl * su;
            dy[8 + b] = sigma * dl * sv;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Fehlberg RKF45 (Sec. 2.3, Fehlberg 1969 coefficients)               */

static const double FA[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
static const double FB4[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
static const double FB5[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0,
                              2.0 / 55.0};
/* Kutta's 3/8 rule (R18) */
static const double K38A[4][3] = {{0, 0, 0}, {1.0 / 3.0, 0, 0}, {-1.0 / 3.0, 1.0, 0}, {1.0, -1.0, 1.0}};
static const double K38B[4] = {1.0 / 8.0, 3.0 / 8.0, 3.0 / 8.0, 1.0 / 8.0};

/* One RKF45 step of size h from y (D: see o_rhs). With haxis >= 0 the
 * independent variable is y[haxis] (Henon step, R5): the RHS is divided by its
 * haxis component, which must be >= graze in the outward direction hsign at
 * every stage.
 * Returns 0 ok, 1 null field, 2 grazing. y5 may be NULL. */
static int o_rkf45(const OField *f, const OParams *p, const double *D, double sigma, int ns, int haxis,
                   double hsign, const double *y, double h, double *y4, double *y5)
{
    double k[6][NSTATE], ys[NSTATE];
    const int rk38 = p->scheme == 1;  /* R18: the 3/8 rule, 4 stages, no error estimate */
    const int nst = rk38 ? 4 : 6;
    for (int s = 0; s < nst; s++) {
        for (int c = 0; c < ns; c++) {
            double acc = 0.0;
            for (int r = 0; r < s; r++) acc += (rk38 ? K38A[s][r] : FA[s][r]) * k[r][c];
            ys[c] = y[c] + h * acc;
        }
        if (o_rhs(f, p, D, sigma, ns, ys, k[s])) return 1;
        if (haxis >= 0) {
            double fa = k[s][haxis];
            double fn = f->X[0] ? fa / D[haxis] : fa; /* in cells per unit tau (R16) */
            if (!(fn * hsign >= p->graze)) return 2;
            for (int c = 0; c < ns; c++) k[s][c] = k[s][c] / fa;
        }
    }
    for (int c = 0; c < ns; c++) {
        double a4 = 0.0, a5 = 0.0;
        if (rk38) {
            for (int s = 0; s < 4; s++) a4 += K38B[s] * k[s][c];
            y4[c] = y[c] + h * a4;
            if (y5) y5[c] = y4[c];
            continue;
        }
        for (int s = 0; s < 6; s++) {
            a4 += FB4[s] * k[s][c];
            a5 += FB5[s] * k[s][c];
        }
        y4[c] = y[c] + h * a4;
        if (y5) y5[c] = y[c] + h * a5;
    }
    return 0;
}

/* the box in state coordinates: [0, n-1] cells, or [x_0, x_{n-1}] (R16) */
static double o_lo(const OField *f, int a) { return f->X[a] ? f->X[a][0] : 0.0; }
static double o_hi(const OField *f, int a) { return f->X[a] ? f->X[a][f->n[a] - 1] : (double)(f->n[a] - 1); }

static int o_inside(const OField *f, const double *xi)
{
    for (int a = 0; a < 3; a++)
        if (!(xi[a] >= o_lo(f, a) && xi[a] <= o_hi(f, a))) return 0;
    return 1;
}

static double o_face_value(const OField *f, int face) { return (face & 1) ? o_hi(f, face >> 1) : o_lo(f, face >> 1); }

/* widths of the cell holding y (the spacing on a uniform grid) */
static void o_widths(const OField *f, const double *y, double D[3])
{
    for (int a = 0; a < 3; a++) {
        if (f->X[a]) {
            long long c = o_cell_rect(f->X[a], f->n[a], y[a]);
            D[a] = f->X[a][c + 1] - f->X[a][c];
        } else {
            D[a] = f->d[a];
        }
    }
}

/* state <-> physical coordinates */
static double o_phys(const OField *f, const double *y, int a) { return f->X[a] ? y[a] : f->o[a] + f->d[a] * y[a]; }
static double o_state(const OField *f, const double *r, int a) { return f->X[a] ? r[a] : (r[a] - f->o[a]) / f->d[a]; }

/* face first crossed by the chord from y (inside) to yn (outside); t = chord parameter */
static int o_chord_face(const OField *f, const double *y, const double *yn, double *tout)
{
    int best = -1;
    double tb = INFINITY;
    for (int a = 0; a < 3; a++) {
        double lo = o_lo(f, a), hi = o_hi(f, a), t;
        int fc;
        if (yn[a] < lo) {
            t = (lo - y[a]) / (yn[a] - y[a]);
            fc = 2 * a;
        } else if (yn[a] > hi) {
            t = (hi - y[a]) / (yn[a] - y[a]);
            fc = 2 * a + 1;
        } else {
            continue;
        }
        if (t < tb) {
            tb = t;
            best = fc;
        }
    }
    *tout = tb;
    return best;
}

/* Trace one direction from the seed state; writes the end state and face.
 * tol: the line's tolerance, or with the fixed-step scheme its step (R18).
 * Returns nonzero when the line must stop with a bad status. */
static int o_trace_dir(const OField *f, const OParams *p, double tol, double sigma, int ns, const double *yseed,
                       double *yend, int *face, long long *steps, int *status, OLog *log)
{
    o_log(log, sigma, 99);
    double y[NSTATE], y4[NSTATE], y5[NSTATE], yt[NSTATE], D[3];
    memcpy(y, yseed, sizeof(double) * ns);
    double h = p->scheme == 1 ? tol : p->h0;
    *face = -1;
    for (;;) {
        if (*steps >= p->max_steps) {
            *status |= ST_MAXSTEPS;
            memcpy(yend, y, sizeof(double) * ns);
            return 1;
        }
        (*steps)++;
        o_widths(f, y, D);
        if (o_rkf45(f, p, D, sigma, ns, -1, 0.0, y, h, y4, y5)) {
            *status |= ST_NULL;
            memcpy(yend, y, sizeof(double) * ns);
            return 1;
        }
        double hn = h; /* the fixed step (R18) */
        if (p->scheme != 1) {
            double e2 = 0.0;
            if (f->X[0]) {
                for (int a = 0; a < 3; a++) e2 += ((y5[a] - y4[a]) / D[a]) * ((y5[a] - y4[a]) / D[a]);
            } else {
                for (int a = 0; a < 3; a++) e2 += (y5[a] - y4[a]) * (y5[a] - y4[a]);
            }
            double err = sqrt(e2);
            if (err > tol) {
                if (h > p->hmin) {
                    h = h * fmax(0.1, 0.9 * sqrt(sqrt(tol / err)));
                    if (h < p->hmin) h = p->hmin;
                    continue;
                }
                *status |= ST_STALL;
            }
            hn = (err > 0.0) ? h * fmin(4.0, 0.9 * sqrt(sqrt(tol / err))) : 4.0 * h;
            if (hn < p->hmin) hn = p->hmin;
            if (hn > p->hmax) hn = p->hmax;
        }
        if (o_inside(f, y4)) {
            o_log(log, h, 0);
            memcpy(y, y4, sizeof(double) * ns);
            h = hn;
            continue;
        }
        /* the accepted step left the box: Henon step onto the exit face (R5) */
        double t0;
        int fc0 = o_chord_face(f, y, y4, &t0);
        int fc = fc0, graze = 0;
        for (int tries = 0;; tries++) {
            int a = fc >> 1;
            double target = o_face_value(f, fc), hsign = (fc & 1) ? 1.0 : -1.0;
            (*steps)++;
            int r = o_rkf45(f, p, D, sigma, ns, a, hsign, y, target - y[a], yt, NULL);
            if (r == 1) {
                *status |= ST_NULL;
                memcpy(yend, y, sizeof(double) * ns);
                return 1;
            }
            if (r == 2) {
                graze = 1;
                break;
            }
            yt[a] = target;
            int nf = -1;
            for (int b = 0; b < 3 && nf < 0; b++) {
                if (b == a) continue;
                if (yt[b] < o_lo(f, b)) nf = 2 * b;
                else if (yt[b] > o_hi(f, b)) nf = 2 * b + 1;
            }
            if (nf < 0) {
                o_log(log, 0.0, 16 + fc);
                memcpy(yend, yt, sizeof(double) * ns);
                *face = fc;
                return 0;
            }
            if (tries >= 2) {
                for (int b = 0; b < 3; b++) {
                    if (yt[b] < o_lo(f, b)) yt[b] = o_lo(f, b);
                    if (yt[b] > o_hi(f, b)) yt[b] = o_hi(f, b);
                }
                o_log(log, 0.0, 40 + fc);
                memcpy(yend, yt, sizeof(double) * ns);
                *face = fc;
                return 0;
            }
            fc = nf;
        }
        if (graze) {
            if (0.5 * h >= p->hmin) {
                h = 0.5 * h;
                continue;
            }
            for (int c = 0; c < ns; c++) yend[c] = y[c] + t0 * (y4[c] - y[c]);
            yend[fc0 >> 1] = o_face_value(f, fc0);
            o_log(log, h, 48 + fc0);
            *face = fc0;
            *status |= ST_CHORD;
            return 0;
        }
    }
}

/* Trace the whole line through physical seed r0. End 1 is the footpoint on the
 * -n0 side of S0 (reached along -s0 B with s0 = sign(B(r0) . n0), +1 when the
 * product is 0 or n0 is NULL), end 2 the other one; end 1 is traced first.
 * U0/V0 may be NULL. */
static void o_trace_line_log(const OField *f, const OParams *p, const double r0[3], const double *n0, double tol,
                             const double *U0, const double *V0, OLine *L, OLog *log, double *s0out)
{
    int ns = (U0 && V0) ? NSTATE : 5;
    double y0[NSTATE];
    memset(L, 0, sizeof *L);
    L->face[0] = L->face[1] = -1;
    for (int a = 0; a < 3; a++) y0[a] = o_state(f, r0, a);
    y0[3] = 0.0;
    y0[4] = 0.0;
    if (ns == NSTATE)
        for (int a = 0; a < 3; a++) {
            y0[5 + a] = U0[a];
            y0[8 + a] = V0[a];
        }
    for (int e = 0; e < 2; e++) memcpy(L->end[e], y0, sizeof(double) * NSTATE);
    if (!o_inside(f, y0)) {
        L->status |= ST_OUTSIDE;
        return;
    }
    double dy[NSTATE], D0[3];
    o_widths(f, y0, D0);
    if (o_rhs(f, p, D0, 1.0, ns, y0, dy)) {
        L->status |= ST_NULL;
        return;
    }
    double s0 = 1.0;
    if (n0) {
        double B0[3];
        o_interp(f, f->B, 3, y0, B0);
        if (B0[0] * n0[0] + B0[1] * n0[1] + B0[2] * n0[2] < 0.0) s0 = -1.0;
    }
    if (s0out) *s0out = s0;
    if (o_trace_dir(f, p, tol, -s0, ns, y0, L->end[0], &L->face[0], &L->steps, &L->status, log)) return;
    if (o_trace_dir(f, p, tol, +s0, ns, y0, L->end[1], &L->face[1], &L->steps, &L->status, log)) return;
    for (int e = 0; e < 2; e++) o_interp(f, f->B, 3, L->end[e], L->Bend[e]);
}

static void o_trace_line(const OField *f, const OParams *p, const double r0[3], const double *n0, double tol,
                         const double *U0, const double *V0, OLine *L)
{
    o_trace_line_log(f, p, r0, n0, tol, U0, V0, L, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* S0 frames and Q assembly                                             */

static double o_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void o_cross(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Rotated S0 (R9): orthonormal u, v perpendicular to bhat */
static void o_perp_frame(const double bh[3], double u[3], double v[3])
{
    int m = 0;
    for (int a = 1; a < 3; a++)
        if (fabs(bh[a]) < fabs(bh[m])) m = a;
    double e[3] = {0, 0, 0}, t[3];
    e[m] = 1.0;
    o_cross(bh, e, t);
    double nt = sqrt(o_dot(t, t));
    for (int a = 0; a < 3; a++) u[a] = t[a] / nt;
    o_cross(bh, u, v);
}

static void o_face_coords(const OField *f, const double *xi, int face, double fc[2])
{
    int a = face >> 1, k = 0;
    for (int b = 0; b < 3; b++)
        if (b != a) fc[k++] = o_phys(f, xi, b);
}

static int o_line_ok(const OLine *L) { return L && !(L->status & ST_BAD); }

/* Method I (R8): nb = {+u, -u, +v, -v} neighbour lines (NULL when off-lattice) */
static double o_q_method1(const OField *f, const OLine *c, const OLine *nb[4], double du, double dv, double bn0,
                          int *status)
{
    double Jm[2][2][2];
    for (int e = 0; e < 2; e++) {
        double f0[2], fp[2], fm[2];
        o_face_coords(f, c->end[e], c->face[e], f0);
        for (int s = 0; s < 2; s++) {
            const OLine *P = nb[2 * s], *M = nb[2 * s + 1];
            double del = s ? dv : du;
            int okp = o_line_ok(P) && P->face[e] == c->face[e];
            int okm = o_line_ok(M) && M->face[e] == c->face[e];
            if (okp) o_face_coords(f, P->end[e], P->face[e], fp);
            if (okm) o_face_coords(f, M->end[e], M->face[e], fm);
            for (int r = 0; r < 2; r++) {
                if (okp && okm) Jm[e][r][s] = (fp[r] - fm[r]) / (2.0 * del);
                else if (okp) Jm[e][r][s] = (fp[r] - f0[r]) / del;
                else if (okm) Jm[e][r][s] = (f0[r] - fm[r]) / del;
                else {
                    *status |= ST_MIXED;
                    return NAN;
                }
            }
        }
    }
    /* Eq. D+-2 with Eq. D+-3: D12 = J2 adj(J1) / |Bn0/Bn1| */
    double adj[2][2] = {{Jm[0][1][1], -Jm[0][0][1]}, {-Jm[0][1][0], Jm[0][0][0]}};
    double norm2 = 0.0;
    for (int r = 0; r < 2; r++)
        for (int s = 0; s < 2; s++) {
            double m = Jm[1][r][0] * adj[0][s] + Jm[1][r][1] * adj[1][s];
            norm2 += m * m;
        }
    double bn1 = c->Bend[0][c->face[0] >> 1], bn2 = c->Bend[1][c->face[1] >> 1];
    /* Eq. Q+- with |det D| -> |Bn1/Bn2| (Eq. Bn1) */
    return norm2 * fabs(bn1 * bn2) / (bn0 * bn0);
}

/* Method II (R10, Eq. q_scott) from the deviation vectors at both ends;
 * perp: Q_perp (R17), the end planes perpendicular to B */
static double o_q_method2(const OLine *c, double bn0, int perp)
{
    double Ut[2][3], Vt[2][3], bn[2];
    for (int e = 0; e < 2; e++) {
        int a = c->face[e] >> 1;
        const double *U = c->end[e] + 5, *V = c->end[e] + 8, *B = c->Bend[e];
        if (perp) {
            double BB = o_dot(B, B), ub = o_dot(U, B) / BB, vb = o_dot(V, B) / BB;
            bn[e] = sqrt(BB);
            for (int b = 0; b < 3; b++) {
                Ut[e][b] = U[b] - ub * B[b];
                Vt[e][b] = V[b] - vb * B[b];
            }
            continue;
        }
        bn[e] = B[a];
        for (int b = 0; b < 3; b++) {
            Ut[e][b] = U[b] - U[a] / B[a] * B[b];
            Vt[e][b] = V[b] - V[a] / B[a] * B[b];
        }
    }
    double num = o_dot(Ut[0], Ut[0]) * o_dot(Vt[1], Vt[1]) + o_dot(Ut[1], Ut[1]) * o_dot(Vt[0], Vt[0]) -
                 2.0 * o_dot(Ut[0], Vt[0]) * o_dot(Ut[1], Vt[1]);
    return fabs(num) * fabs(bn[0] * bn[1]) / (bn0 * bn0);
}

/* ------------------------------------------------------------------ */
/* lattices (R7) and the public entry points                           */

typedef struct {
    double o[3], a1[3], a2[3], a3[3];
    long long n1, n2, n3;
} OLattice;

static void o_seed(const OLattice *L, long long i, long long j, long long k, double r[3])
{
    for (int a = 0; a < 3; a++)
        r[a] = L->o[a] + (i + 0.5) * L->a1[a] + (j + 0.5) * L->a2[a] + (k + 0.5) * L->a3[a];
}

/* 1 if the layer through r with normal n0 lies on a face of the box */
static int o_on_face(const OField *f, const double n0[3], const double r[3])
{
    int axis = -1, zeros = 0;
    for (int a = 0; a < 3; a++) {
        if (n0[a] == 0.0) zeros++;
        else axis = a;
    }
    if (zeros != 2) return 0;
    double xi = o_state(f, r, axis);
    return xi == o_lo(f, axis) || xi == o_hi(f, axis);
}

typedef struct {
    double r0[3], n0[3], bh[3], u[3], v[3];
    double bn0, bn0s, tol; /* Bn0 used by Q, signed B0.n0; tol: the line's tolerance or step (R18) */
    int rotated, bad;
} OSeed;

/* the tolerance (RKF45) or step (3/8 rule) of a line in the perpendicular case */
static double o_ctl_perp(const OParams *p) { return p->scheme == 1 ? p->step : p->tol; }

/* S0 frame and tolerance of one lattice seed (R9, R10) */
static void o_seed_setup(const OField *f, const OParams *p, const OLattice *L, long long i, long long j,
                         long long k, OSeed *S)
{
    memset(S, 0, sizeof *S);
    o_seed(L, i, j, k, S->r0);
    double nn[3];
    o_cross(L->a1, L->a2, nn);
    double m = sqrt(o_dot(nn, nn));
    for (int a = 0; a < 3; a++) S->n0[a] = nn[a] / m;
    double xi[3], B[3];
    for (int a = 0; a < 3; a++) xi[a] = o_state(f, S->r0, a);
    if (!o_inside(f, xi)) {
        S->bad = ST_OUTSIDE;
        return;
    }
    o_interp(f, f->B, 3, xi, B);
    double nB = sqrt(o_dot(B, B));
    if (!(nB > 0) || !isfinite(nB)) {
        S->bad = ST_NULL;
        return;
    }
    for (int a = 0; a < 3; a++) S->bh[a] = B[a] / nB;
    S->bn0s = o_dot(B, S->n0);
    o_perp_frame(S->bh, S->u, S->v);
    if (p->method == 2) {
        S->bn0 = nB;
        S->tol = o_ctl_perp(p);
        return;
    }
    double ratio = fabs(o_dot(B, S->n0)) / nB;
    if (ratio < p->rot_thresh && !o_on_face(f, S->n0, S->r0)) {
        S->rotated = 1;
        S->bn0 = nB;
        S->tol = o_ctl_perp(p);
    } else {
        S->bn0 = o_dot(B, S->n0);
        if (p->scheme == 1) {
            S->tol = fmax(p->step * ratio, p->step_min); /* Eq. step (R18) */
        } else {
            double x = fmax(ratio, p->rot_thresh);
            S->tol = p->tol * (p->tol_exp == 1.5 ? x * sqrt(x) : pow(x, p->tol_exp));
        }
    }
}

static void o_write(const OField *f, const OLine *c, long long s, double Q, double *Qo, double *Two, double *leno,
                    double *r1, double *r2, int *f1, int *f2, int *st, long long *steps)
{
    int bad = c->status & ST_BAD;
    if (Qo) Qo[s] = (bad || (c->status & ST_MIXED)) ? NAN : Q;
    if (Two) Two[s] = bad ? NAN : c->end[0][4] + c->end[1][4];
    if (leno) leno[s] = bad ? NAN : c->end[0][3] + c->end[1][3];
    for (int a = 0; a < 3; a++) {
        if (r1) r1[3 * s + a] = o_phys(f, c->end[0], a);
        if (r2) r2[3 * s + a] = o_phys(f, c->end[1], a);
    }
    if (f1) f1[s] = c->face[0];
    if (f2) f2[s] = c->face[1];
    if (st) st[s] = c->status;
    if (steps) steps[s] = c->steps;
}

static int o_make_field(OField *f, const double *B, const double *J, const double *G, const long long n[3],
                        const double o[3], const double d[3])
{
    for (int a = 0; a < 3; a++) {
        if (n[a] < 2 || !(d[a] > 0)) return 1;
        f->n[a] = n[a];
        f->o[a] = o[a];
        f->d[a] = d[a];
    }
    f->B = B;
    f->J = J;
    f->G = G;
    f->X[0] = f->X[1] = f->X[2] = NULL;
    return 0;
}

/* stretched grid (R16): X = x, y, z node coordinates back to back, each
 * strictly increasing */
static int o_make_field_rect(OField *f, const double *B, const double *J, const double *G, const long long n[3],
                             const double *X)
{
    long long off = 0;
    for (int a = 0; a < 3; a++) {
        if (n[a] < 2) return 1;
        f->n[a] = n[a];
        f->X[a] = X + off;
        for (long long i = 0; i + 1 < n[a]; i++)
            if (!(f->X[a][i + 1] > f->X[a][i])) return 1;
        f->o[a] = f->X[a][0];
        f->d[a] = NAN; /* not used on a stretched grid */
        off += n[a];
    }
    f->B = B;
    f->J = J;
    f->G = G;
    return 0;
}

/* Q, Tw, length, footpoints, faces, status and step counts on a seed lattice.
 * ln = {n1, n2, n3}; a3 = 0 and n3 = 1 for a plane. sample = linear lattice
 * indices (i + n1 (j + n2 k)) to compute, or NULL for the whole lattice. */
static int o_qmap(const OField *fp, const double lo[3], const double a1[3], const double a2[3], const double a3[3],
                  const long long ln[3], const OParams *p, const long long *sample, long long nsample, double *Qo,
                  double *Two, double *leno, double *r1, double *r2, int *f1, int *f2, int *st, long long *steps);

int oracle_qmap(const double *B, const double *J, const double *G, const long long n[3], const double o[3],
                const double d[3], const double lo[3], const double a1[3], const double a2[3], const double a3[3],
                const long long ln[3], const OParams *p, const long long *sample, long long nsample, double *Qo,
                double *Two, double *leno, double *r1, double *r2, int *f1, int *f2, int *st, long long *steps)
{
    OField f;
    if (o_make_field(&f, B, J, G, n, o, d)) return 1;
    if (p->method == 2 && p->way == 1 && !G) return 2;
    return o_qmap(&f, lo, a1, a2, a3, ln, p, sample, nsample, Qo, Two, leno, r1, r2, f1, f2, st, steps);
}

/* The same on a stretched grid (R16). */
int oracle_qmap_rect(const double *B, const double *J, const double *G, const long long n[3], const double *X,
                     const double lo[3], const double a1[3], const double a2[3], const double a3[3],
                     const long long ln[3], const OParams *p, const long long *sample, long long nsample, double *Qo,
                     double *Two, double *leno, double *r1, double *r2, int *f1, int *f2, int *st, long long *steps)
{
    OField f;
    if (o_make_field_rect(&f, B, J, G, n, X)) return 1;
    if (p->method == 2 && p->way == 1 && !G) return 2;
    return o_qmap(&f, lo, a1, a2, a3, ln, p, sample, nsample, Qo, Two, leno, r1, r2, f1, f2, st, steps);
}

static int o_qmap(const OField *fp, const double lo[3], const double a1[3], const double a2[3], const double a3[3],
                  const long long ln[3], const OParams *p, const long long *sample, long long nsample, double *Qo,
                  double *Two, double *leno, double *r1, double *r2, int *f1, int *f2, int *st, long long *steps)
{
    const OField f = *fp;
    OLattice L;
    for (int a = 0; a < 3; a++) {
        L.o[a] = lo[a];
        L.a1[a] = a1[a];
        L.a2[a] = a2[a];
        L.a3[a] = a3[a];
    }
    L.n1 = ln[0];
    L.n2 = ln[1];
    L.n3 = ln[2];
    if (L.n1 < 1 || L.n2 < 1 || L.n3 < 1) return 3;
    double du = sqrt(o_dot(a1, a1)), dv = sqrt(o_dot(a2, a2)), drot = fmin(du, dv);
    long long total = L.n1 * L.n2 * L.n3;
    long long count = sample ? nsample : total;

#pragma omp parallel for schedule(dynamic, 4)
    for (long long s = 0; s < count; s++) {
        long long idx = sample ? sample[s] : s;
        long long i = idx % L.n1, j = (idx / L.n1) % L.n2, k = idx / (L.n1 * L.n2);
        OSeed S;
        OLine c;
        o_seed_setup(&f, p, &L, i, j, k, &S);
        if (S.bad) {
            memset(&c, 0, sizeof c);
            c.face[0] = c.face[1] = -1;
            c.status = S.bad;
            for (int e = 0; e < 2; e++)
                for (int a = 0; a < 3; a++) c.end[e][a] = o_state(&f, S.r0, a);
            o_write(&f, &c, s, NAN, Qo, Two, leno, r1, r2, f1, f2, st, steps);
            continue;
        }
        double Q;
        if (p->method == 2) {
            o_trace_line(&f, p, S.r0, S.n0, S.tol, S.u, S.v, &c);
            Q = o_q_method2(&c, S.bn0, p->qperp);
        } else {
            o_trace_line(&f, p, S.r0, S.n0, S.tol, NULL, NULL, &c);
            OLine nbl[4];
            const OLine *nb[4] = {NULL, NULL, NULL, NULL};
            if (S.rotated) {
                c.status |= ST_ROTATED;
                /* the extra lines are ordered like the centre: n = sign(B0.n0) bhat */
                double nrot[3];
                for (int a = 0; a < 3; a++) nrot[a] = (S.bn0s < 0.0 ? -1.0 : 1.0) * S.bh[a];
                for (int q = 0; q < 4; q++) {
                    const double *dir = (q < 2) ? S.u : S.v;
                    double sg = (q & 1) ? -1.0 : 1.0, rr[3];
                    for (int a = 0; a < 3; a++) rr[a] = S.r0[a] + sg * drot * dir[a];
                    o_trace_line(&f, p, rr, nrot, o_ctl_perp(p), NULL, NULL, &nbl[q]);
                    nb[q] = &nbl[q];
                }
                Q = o_line_ok(&c) ? o_q_method1(&f, &c, nb, drot, drot, S.bn0, &c.status) : NAN;
            } else {
                long long ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
                for (int q = 0; q < 4; q++) {
                    if (ni[q] < 0 || ni[q] >= L.n1 || nj[q] < 0 || nj[q] >= L.n2) continue;
                    OSeed SN;
                    o_seed_setup(&f, p, &L, ni[q], nj[q], k, &SN);
                    if (SN.bad) continue;
                    o_trace_line(&f, p, SN.r0, SN.n0, SN.tol, NULL, NULL, &nbl[q]);
                    nb[q] = &nbl[q];
                }
                Q = o_line_ok(&c) ? o_q_method1(&f, &c, nb, du, dv, S.bn0, &c.status) : NAN;
            }
        }
        o_write(&f, &c, s, Q, Qo, Two, leno, r1, r2, f1, f2, st, steps);
    }
    return 0;
}

/* Tw, length and footpoints for an explicit list of physical seeds (no Q). */
static int o_twist(const OField *fp, const double *seeds, long long ns, const OParams *p, double *Two, double *leno,
                   double *r1, double *r2, int *f1, int *f2, int *st, long long *steps)
{
    const OField f = *fp;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long s = 0; s < ns; s++) {
        OLine c;
        o_trace_line(&f, p, seeds + 3 * s, NULL, o_ctl_perp(p), NULL, NULL, &c);
        o_write(&f, &c, s, NAN, NULL, Two, leno, r1, r2, f1, f2, st, steps);
    }
    return 0;
}

int oracle_twist(const double *B, const double *J, const long long n[3], const double o[3], const double d[3],
                 const double *seeds, long long ns, const OParams *p, double *Two, double *leno, double *r1,
                 double *r2, int *f1, int *f2, int *st, long long *steps)
{
    OField f;
    if (o_make_field(&f, B, J, NULL, n, o, d)) return 1;
    return o_twist(&f, seeds, ns, p, Two, leno, r1, r2, f1, f2, st, steps);
}

/* Tw, length and footpoints on a stretched grid (R16). */
int oracle_twist_rect(const double *B, const double *J, const long long n[3], const double *X, const double *seeds,
                      long long ns, const OParams *p, double *Two, double *leno, double *r1, double *r2, int *f1,
                      int *f2, int *st, long long *steps)
{
    OField f;
    if (o_make_field_rect(&f, B, J, NULL, n, X)) return 1;
    return o_twist(&f, seeds, ns, p, Two, leno, r1, r2, f1, f2, st, steps);
}

/* Trilinear interpolation (Eqs. interp, w0, w1) on a stretched grid at
 * physical points r (np x 3). */
int oracle_interp_rect(const double *arr, int nc, const long long n[3], const double *X, const double *r,
                       long long np, double *out)
{
    OField f;
    memset(&f, 0, sizeof f);
    if (o_make_field_rect(&f, arr, NULL, NULL, n, X)) return 1;
    for (long long k = 0; k < np; k++) o_interp(&f, arr, nc, r + 3 * k, out + (long long)nc * k);
    return 0;
}

/* Cell index of each coordinate on one stretched axis (for tests). */
int oracle_cell_rect(const double *X, long long n, const double *x, long long m, long long *out)
{
    if (n < 2) return 1;
    for (long long k = 0; k < m; k++) out[k] = o_cell_rect(X, n, x[k]);
    return 0;
}

/* Raw line tracing for tests: per-line tol, optional deviation vectors U0/V0
 * (n x 3 each). Outputs the end states (n x 2 x 11), faces (n x 2), end B
 * (n x 2 x 3), status and steps. */
int oracle_trace(const double *B, const double *J, const double *G, const long long n[3], const double o[3],
                 const double d[3], const double *seeds, long long ns, const double *tol, const double *U0,
                 const double *V0, const OParams *p, double *ends, int *faces, double *Bend, int *st,
                 long long *steps)
{
    OField f;
    if (o_make_field(&f, B, J, G, n, o, d)) return 1;
    if (U0 && p->way == 1 && !G) return 2;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long s = 0; s < ns; s++) {
        OLine c;
        o_trace_line(&f, p, seeds + 3 * s, NULL, tol[s], U0 ? U0 + 3 * s : NULL, V0 ? V0 + 3 * s : NULL, &c);
        memcpy(ends + s * 2 * NSTATE, c.end, sizeof c.end);
        memcpy(Bend + s * 6, c.Bend, sizeof c.Bend);
        faces[2 * s] = c.face[0];
        faces[2 * s + 1] = c.face[1];
        st[s] = c.status;
        steps[s] = c.steps;
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Lines of a plane lattice traced once, with the record of their accepted
 * steps (OLog codes; at most cap entries per line, logn[s] = -1 on overflow),
 * orientation sign s0, tolerance, Bn0, end states (s x 2 x 11), faces and
 * status: every seed (which = NULL; output s = lattice index), or the nwhich
 * lattice indices which[] (output s = position in which). For a seed whose S0
 * is rotated, the four extra lines (+u, -u, +v, -v of the rotated frame) are
 * traced as the Q map traces them and, if xlogh is not NULL, recorded in the
 * x* arrays (4 per seed: records of cap entries, counts, s0, faces (2),
 * status). Used by the adjoint tests to replay the frozen step sequence. */
static int o_lattice_log(const OField *pf, const double lo[3], const double a1[3], const double a2[3],
                         const long long ln[2], const OParams *p, int cap, double *logh, int *logc, int *logn,
                         double *s0o, double *tolo, double *bn0o, double *ends, int *faces, int *st,
                         const long long *which, long long nwhich, double *xlogh, int *xlogc, int *xlogn, double *xs0,
                         int *xfaces, int *xst)
{
    OField f = *pf;
    if (p->method != 1) return 2;
    OLattice L;
    for (int a = 0; a < 3; a++) {
        L.o[a] = lo[a];
        L.a1[a] = a1[a];
        L.a2[a] = a2[a];
        L.a3[a] = 0.0;
    }
    L.n1 = ln[0];
    L.n2 = ln[1];
    L.n3 = 1;
    long long total = which ? nwhich : L.n1 * L.n2;
    if (which)
        for (long long s = 0; s < nwhich; s++)
            if (which[s] < 0 || which[s] >= L.n1 * L.n2) return 3;
#pragma omp parallel for schedule(dynamic, 4)
    for (long long s = 0; s < total; s++) {
        long long idx = which ? which[s] : s;
        long long i = idx % L.n1, j = idx / L.n1;
        OSeed S;
        OLine c;
        OLog g = {logh + s * cap, logc + s * cap, cap, 0, 0};
        double s0 = 1.0;
        o_seed_setup(&f, p, &L, i, j, 0, &S);
        memset(&c, 0, sizeof c);
        c.face[0] = c.face[1] = -1;
        if (S.bad) {
            c.status = S.bad;
        } else {
            o_trace_line_log(&f, p, S.r0, S.n0, S.tol, NULL, NULL, &c, &g, &s0);
            if (S.rotated) c.status |= ST_ROTATED;
        }
        logn[s] = g.overflow ? -1 : g.n;
        if (xlogh) {
            for (int q = 0; q < 4; q++) {
                xlogn[4 * s + q] = 0;
                xs0[4 * s + q] = 1.0;
                xfaces[8 * s + 2 * q] = xfaces[8 * s + 2 * q + 1] = -1;
                xst[4 * s + q] = 0;
            }
            if (!S.bad && S.rotated) {
                /* the extra lines as the Q map traces them (ordered like the centre) */
                const double du = sqrt(o_dot(a1, a1)), dv = sqrt(o_dot(a2, a2)), drot = fmin(du, dv);
                double nrot[3];
                for (int a = 0; a < 3; a++) nrot[a] = (S.bn0s < 0.0 ? -1.0 : 1.0) * S.bh[a];
                for (int q = 0; q < 4; q++) {
                    const double *dir = (q < 2) ? S.u : S.v;
                    double sg = (q & 1) ? -1.0 : 1.0, rr[3], sx = 1.0;
                    for (int a = 0; a < 3; a++) rr[a] = S.r0[a] + sg * drot * dir[a];
                    OLine xl;
                    OLog gx = {xlogh + (4 * s + q) * (long long)cap, xlogc + (4 * s + q) * (long long)cap, cap, 0, 0};
                    o_trace_line_log(&f, p, rr, nrot, o_ctl_perp(p), NULL, NULL, &xl, &gx, &sx);
                    xlogn[4 * s + q] = gx.overflow ? -1 : gx.n;
                    xs0[4 * s + q] = sx;
                    xfaces[8 * s + 2 * q] = xl.face[0];
                    xfaces[8 * s + 2 * q + 1] = xl.face[1];
                    xst[4 * s + q] = xl.status;
                }
            }
        }
        s0o[s] = s0;
        tolo[s] = S.tol;
        bn0o[s] = S.bn0;
        memcpy(ends + s * 2 * NSTATE, c.end, sizeof c.end);
        faces[2 * s] = c.face[0];
        faces[2 * s + 1] = c.face[1];
        st[s] = c.status;
    }
    return 0;
}

/* The step record of every lattice line (R13), uniform grid. */
int oracle_lattice_log(const double *B, const double *J, const long long n[3], const double o[3], const double d[3],
                       const double lo[3], const double a1[3], const double a2[3], const long long ln[2],
                       const OParams *p, int cap, double *logh, int *logc, int *logn, double *s0o, double *tolo,
                       double *bn0o, double *ends, int *faces, int *st, const long long *which, long long nwhich,
                       double *xlogh, int *xlogc, int *xlogn, double *xs0, int *xfaces, int *xst)
{
    OField f;
    if (o_make_field(&f, B, J, NULL, n, o, d)) return 1;
    return o_lattice_log(&f, lo, a1, a2, ln, p, cap, logh, logc, logn, s0o, tolo, bn0o, ends, faces, st, which,
                         nwhich, xlogh, xlogc, xlogn, xs0, xfaces, xst);
}

/* The same on a stretched grid (R16; X = the nx + ny + nz node coordinates):
 * the recorded ends are physical positions. */
int oracle_lattice_log_rect(const double *B, const double *J, const long long n[3], const double *X,
                            const double lo[3], const double a1[3], const double a2[3], const long long ln[2],
                            const OParams *p, int cap, double *logh, int *logc, int *logn, double *s0o, double *tolo,
                            double *bn0o, double *ends, int *faces, int *st, const long long *which, long long nwhich,
                            double *xlogh, int *xlogc, int *xlogn, double *xs0, int *xfaces, int *xst)
{
    OField f;
    if (o_make_field_rect(&f, B, J, NULL, n, X)) return 1;
    return o_lattice_log(&f, lo, a1, a2, ln, p, cap, logh, logc, logn, s0o, tolo, bn0o, ends, faces, st, which,
                         nwhich, xlogh, xlogc, xlogn, xs0, xfaces, xst);
}
