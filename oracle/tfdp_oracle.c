/*
 * tfdp_oracle.c -- plain, slow, FP64 CPU oracle for one t-FDP iteration.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check, and the benchmark's
 * CPU-baseline leg and reference arm load this library. The GPU library shares no
 * code with it and never links it.
 *
 * It follows "Force-directed graph layouts revisited: a new force based on the
 * t-Distribution" (Zhong, Xue, Zhang, Zhang, Ban, Deussen, Wang; arXiv 2303.03964):
 *
 *   exact repulsion       Sec. 3.3 Eq. (replusive); Sec. 3.4 Eq. (repfK)
 *   attraction            Sec. 3.3 Eq. (newforce), weighted by alpha as in the
 *                         resultant force of Sec. 3.3
 *   ibFFT repulsion       Sec. 3.4: Lagrange projection onto k x k equispaced nodes in
 *                         each of N_int x N_int boxes over the layout square, grid
 *                         interaction by FFT, back-projection, then Eq. (Fr1)/(Fr2)
 *                         with the three kernel sums of Eq. (kernelproduct)
 *   grid size             Sec. 3.4 "Choices of k": N_int = max(50, [L]). Policy
 *                         GRID_PAPER takes h = L / N_int; GRID_SNAP_H rounds h up to
 *                         2^e (16 + j) / 16 so that the spectrum can be cached. SNAP_H
 *                         is a reading, not the paper's: parity unpinned against the
 *                         paper (the tests pin its arithmetic, not its choice).
 *   dynamic k             Sec. 3.4 "Choices of k": k = 1 for the first 90% of the
 *                         iterations, k = 2 for the next 5%, k = 3 for the rest
 *                         (boundaries floor(0.9 T), floor(0.95 T): a reading)
 *   position update       Sec. 3.1 (move along the resultant force until convergence);
 *                         the step schedule is a reading, the paper gives none: parity
 *                         unpinned against the paper (pinned only by the closed-form
 *                         equilibria the iteration must reach).
 *   local refinement      Sec. 5 "Local Refinement" (fisheye views): stronger attraction
 *                         between focal nodes and their neighbours, stronger repulsion
 *                         elsewhere. The paper gives no formula; the reading is per-node
 *                         weights r_i (repulsion) and a_i (attraction) with the pair
 *                         repulsion scaled by r_i r_j and the edge attraction by a_i a_j,
 *                         which keeps D = -grad E for the weighted energy below. Every
 *                         weight argument may be NULL (all weights 1: the plain method).
 *
 * Sign convention (reading of Sec. 3.3/3.4): the functions return the displacement
 * direction of each node. Repulsion pushes node i away from j,
 *     frep(i) = sum_{j != i} (x_i - x_j) / (1 + |x_i - x_j|^2)^gamma      (Eq. repfK)
 * and attraction pulls it towards its neighbours,
 *     fatt(i) = alpha * sum_{j <-> i} (1 + beta / (1 + d_ij^2)) (x_j - x_i).
 * Their sum D(i) = frep(i) + fatt(i) is minus the gradient of
 *     E = sum_{i<j} (1+d^2)^(1-gamma) / (2(gamma-1))
 *       + alpha * sum_{edges} [ d^2/2 + (beta/2) ln(1+d^2) ].
 * With local-refinement weights: frep(i) = r_i sum_j r_j K_ij (x_i - x_j),
 * fatt(i) = alpha sum_{j <-> i} a_i a_j (...)(x_j - x_i), and each term of E carries the
 * same product of weights.
 *
 * Floating point decides one integer here: the box that holds a node. Both this
 * oracle and the GPU library take that decision in IEEE FP32 with the same
 * operations (see or_box_f32), and take the grid descriptor from exact FP64
 * operations on FP32 extremes, so that both sides use the same boxes.
 * Everything else is FP64.
 *
 * Built with -ffp-contract=off so that the FP32 box decision is not fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* t-force and kernel, Sec. 3.2 Eq. (forcefunction), Sec. 3.4 kernel K.       */
/* ------------------------------------------------------------------------- */

/* K(d^2) = (1 + d^2)^(-gamma), the kernel of Eq. (repfK). */
static double or_kernel(double d2, double gamma) { return pow(1.0 + d2, -gamma); }

/* Local-refinement weight of node i (1 without weights). */
static double or_w(const double* w, int64_t i) { return w ? w[i] : 1.0; }

/* f(d) = d / (1 + d^2)^phi, Eq. (forcefunction). Exposed for the pins. */
double or_tforce(double d, double phi) { return d / pow(1.0 + d * d, phi); }

/* ------------------------------------------------------------------------- */
/* Exact repulsion, Eq. (repfK): rows [i0, i1) of the n x n sum (all sources). */
/* ------------------------------------------------------------------------- */
void or_rep_exact(int64_t n, const double* xy, const double* wr, double gamma, int64_t i0, int64_t i1,
                  double* frep /* 2*(i1-i0) */) {
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = i0; i < i1; ++i) {
        double xi = xy[2 * i], yi = xy[2 * i + 1];
        double fx = 0.0, fy = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - xy[2 * j], dy = yi - xy[2 * j + 1];
            double K = or_w(wr, j) * or_kernel(dx * dx + dy * dy, gamma);
            fx += K * dx;
            fy += K * dy;
        }
        frep[2 * (i - i0)] = or_w(wr, i) * fx;
        frep[2 * (i - i0) + 1] = or_w(wr, i) * fy;
    }
}

/* Same sum for an explicit list of target rows (row-sampled check at large n). */
void or_rep_exact_rows(int64_t n, const double* xy, const double* wr, double gamma, int64_t nrows,
                       const int64_t* rows, double* frep /* 2*nrows */) {
    int64_t r;
#pragma omp parallel for schedule(dynamic, 4)
    for (r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double xi = xy[2 * i], yi = xy[2 * i + 1];
        double fx = 0.0, fy = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = xi - xy[2 * j], dy = yi - xy[2 * j + 1];
            double K = or_w(wr, j) * or_kernel(dx * dx + dy * dy, gamma);
            fx += K * dx;
            fy += K * dy;
        }
        frep[2 * r] = or_w(wr, i) * fx;
        frep[2 * r + 1] = or_w(wr, i) * fy;
    }
}

/* ------------------------------------------------------------------------- */
/* Attraction, Eq. (newforce) times alpha (resultant force, Sec. 3.3).        */
/* edges: m undirected pairs (e[2q], e[2q+1]); each adds to both endpoints.   */
/* ------------------------------------------------------------------------- */
void or_att(int64_t n, int64_t m, const int32_t* edges, const double* xy, const double* wa,
            double alpha, double beta, double* fatt /* 2n */) {
    memset(fatt, 0, sizeof(double) * 2 * (size_t)n);
    for (int64_t q = 0; q < m; ++q) {
        int64_t i = edges[2 * q], j = edges[2 * q + 1];
        double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
        double c = alpha * or_w(wa, i) * or_w(wa, j) * (1.0 + beta / (1.0 + dx * dx + dy * dy));
        fatt[2 * i] += c * dx;
        fatt[2 * i + 1] += c * dy;
        fatt[2 * j] -= c * dx;
        fatt[2 * j + 1] -= c * dy;
    }
}

/* Energy whose negative gradient is frep + fatt (reading of the sign, Sec. 3.3). */
double or_energy(int64_t n, const double* xy, int64_t m, const int32_t* edges, const double* wr,
                 const double* wa, double alpha, double beta, double gamma) {
    double rep = 0.0;
    int64_t i;
#pragma omp parallel for reduction(+ : rep) schedule(dynamic, 16)
    for (i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
            rep += or_w(wr, i) * or_w(wr, j) * pow(1.0 + dx * dx + dy * dy, 1.0 - gamma) / (2.0 * (gamma - 1.0));
        }
    }
    double att = 0.0;
    for (int64_t q = 0; q < m; ++q) {
        int64_t a = edges[2 * q], b = edges[2 * q + 1];
        double dx = xy[2 * a] - xy[2 * b], dy = xy[2 * a + 1] - xy[2 * b + 1];
        double d2 = dx * dx + dy * dy;
        att += or_w(wa, a) * or_w(wa, b) * (0.5 * d2 + 0.5 * beta * log1p(d2));
    }
    return rep + alpha * att;
}

/* ------------------------------------------------------------------------- */
/* Grid policy, Sec. 3.4: the layout square [x_min, x_max]^2 (one interval for */
/* both axes) split into N_int x N_int boxes, N_int = max(50, ceil(L)).        */
/* ------------------------------------------------------------------------- */
enum { OR_GRID_PAPER = 0, OR_GRID_SNAP_H = 1 };

#define OR_L_FLOOR (1.0 / 1024.0)

/*
 * out[0] = lo (FP64 value of the FP32 minimum over both coordinates)
 * out[1] = h  (box side)
 * out[2] = N_int, out[3] = G = N_int * k, out[4] = L
 * Readings: [.] in the N_int rule is the ceiling; N_int is capped at
 * floor(grid_max / k); a layout narrower than 2^-10 is widened to 2^-10.
 * PAPER:  h = L / N_int.
 * SNAP_H: h = the smallest 2^e * (16 + j) / 16 (j = 0..15) with N_int * h >= L, so the
 *         box side, and with it the kernel spectrum, changes only in steps of 1/16 octave.
 */
void or_grid_policy(int64_t n, const float* xyf, int k, int n_int_min, int grid_max, int policy,
                    double* out) {
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = 0; i < 2 * n; ++i) {
        if (xyf[i] < lo) lo = xyf[i];
        if (xyf[i] > hi) hi = xyf[i];
    }
    if (n == 0) { lo = 0.0f; hi = 0.0f; }
    double L = (double)hi - (double)lo;
    if (L < OR_L_FLOOR) L = OR_L_FLOOR;
    double c = ceil(L);
    if (c > 2.0e9) c = 2.0e9; /* keeps the integer conversion defined */
    int n_int = (c > (double)n_int_min) ? (int)c : n_int_min;
    int cap = grid_max / k;
    if (n_int > cap) n_int = cap;
    if (n_int < 1) n_int = 1;
    double h;
    if (policy == OR_GRID_PAPER) {
        h = L / (double)n_int;
    } else {
        int e;
        double t = L / (double)n_int;
        (void)frexp(t, &e); /* t in [2^(e-1), 2^e) */
        double base = ldexp(1.0, e - 1);
        h = ldexp(1.0, e);
        for (int j = 0; j <= 16; ++j) {
            double cand = base * (16.0 + j) / 16.0;
            if ((double)n_int * cand >= L) { h = cand; break; }
        }
    }
    out[0] = (double)lo;
    out[1] = h;
    out[2] = (double)n_int;
    out[3] = (double)(n_int * k);
    out[4] = L;
}

/* Box index along one axis, decided in IEEE FP32: floor((x - lo) / h), clamped to
 * [0, N_int - 1] (a node at x_max goes to the last box). */
int or_box_f32(float x, float lo, float h, int n_int) {
    volatile float d = x - lo;
    volatile float t = d / h;
    float a = floorf(t);
    /* NaN and negative quotients go to box 0, quotients past the end to the last box */
    return (a >= 0.0f) ? ((a <= (float)(n_int - 1)) ? (int)a : n_int - 1) : 0;
}

/* Lagrange basis over the k equispaced nodes t_l = (l + 1/2) / k of a unit box,
 * evaluated at u (box units). k = 1 gives weight 1 at the box centre. */
void or_lagrange(int k, double u, double* w) {
    for (int l = 0; l < k; ++l) {
        double tl = (l + 0.5) / k, v = 1.0;
        for (int q = 0; q < k; ++q) {
            if (q == l) continue;
            double tq = (q + 0.5) / k;
            v *= (u - tq) / (tl - tq);
        }
        w[l] = v;
    }
}

/* ------------------------------------------------------------------------- */
/* Radix-2 FFT (textbook iterative Cooley-Tukey), FP64, in place.             */
/* sign = -1: forward  X_k = sum x_n e^{-2 pi i n k / N}; sign = +1: inverse  */
/* without the 1/N factor.                                                    */
/* ------------------------------------------------------------------------- */
void or_fft(int64_t N, double* re, double* im, int sign) {
    /* w[q] = e^{sign 2 pi i q / N}; stage `len` uses w[q N / len] (same angle). */
    double* wr_t = (double*)malloc(sizeof(double) * (size_t)(N / 2 + 1));
    double* wi_t = (double*)malloc(sizeof(double) * (size_t)(N / 2 + 1));
    for (int64_t q = 0; q < N / 2 + 1; ++q) {
        double ang = sign * 2.0 * OR_PI * (double)q / (double)N;
        wr_t[q] = cos(ang);
        wi_t[q] = sin(ang);
    }
    for (int64_t i = 1, j = 0; i < N; ++i) {
        int64_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int64_t len = 2; len <= N; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t s = 0; s < N; s += len) {
            for (int64_t q = 0; q < half; ++q) {
                double wr = wr_t[q * (N / len)], wi = wi_t[q * (N / len)];
                double ur = re[s + q], ui = im[s + q];
                double vr = re[s + q + half] * wr - im[s + q + half] * wi;
                double vi = re[s + q + half] * wi + im[s + q + half] * wr;
                re[s + q] = ur + vr; im[s + q] = ui + vi;
                re[s + q + half] = ur - vr; im[s + q + half] = ui - vi;
            }
        }
    }
    free(wr_t);
    free(wi_t);
}

/* 2D transform of an N x N row-major array: rows, then columns. */
void or_fft2(int64_t N, double* re, double* im, int sign) {
    int64_t r;
#pragma omp parallel for schedule(static)
    for (r = 0; r < N; ++r) or_fft(N, re + r * N, im + r * N, sign);
#pragma omp parallel
    {
        double* cr = (double*)malloc(sizeof(double) * (size_t)N);
        double* ci = (double*)malloc(sizeof(double) * (size_t)N);
        int64_t c;
#pragma omp for schedule(static)
        for (c = 0; c < N; ++c) {
            for (int64_t q = 0; q < N; ++q) { cr[q] = re[q * N + c]; ci[q] = im[q * N + c]; }
            or_fft(N, cr, ci, sign);
            for (int64_t q = 0; q < N; ++q) { re[q * N + c] = cr[q]; im[q * N + c] = ci[q]; }
        }
        free(cr);
        free(ci);
    }
}

/* ------------------------------------------------------------------------- */
/* Grid interaction, Sec. 3.4 second step: for each of nch channels of a      */
/* G x G grid (row-major, [y][x]) with node spacing s,                         */
/*    out_c[p] = sum_q K(|y_p - y_q|^2) in_c[q],  K = (1 + d^2)^-gamma,        */
/* a linear (non-periodic) convolution. FFT route: embed the kernel in a P x P */
/* circulant, P >= 2G - 1 a power of two, zero-pad the charges, multiply.      */
/* ------------------------------------------------------------------------- */
int or_conv_grid_fft(int64_t G, int64_t P, double s, double gamma, int nch, const double* in,
                     double* out) {
    if (P < 2 * G - 1) return -1;
    size_t PP = (size_t)P * (size_t)P;
    double* kr = (double*)calloc(PP, sizeof(double));
    double* ki = (double*)calloc(PP, sizeof(double));
    double* cr = (double*)malloc(PP * sizeof(double));
    double* ci = (double*)malloc(PP * sizeof(double));
    if (!kr || !ki || !cr || !ci) { free(kr); free(ki); free(cr); free(ci); return -2; }
    for (int64_t dy = -(G - 1); dy <= G - 1; ++dy)
        for (int64_t dx = -(G - 1); dx <= G - 1; ++dx) {
            double d2 = (double)(dx * dx + dy * dy) * s * s;
            int64_t iy = (dy + P) % P, ix = (dx + P) % P;
            kr[iy * P + ix] = or_kernel(d2, gamma);
        }
    or_fft2(P, kr, ki, -1);
    for (int c = 0; c < nch; ++c) {
        memset(cr, 0, PP * sizeof(double));
        memset(ci, 0, PP * sizeof(double));
        for (int64_t y = 0; y < G; ++y)
            for (int64_t x = 0; x < G; ++x) cr[y * P + x] = in[(size_t)c * G * G + y * G + x];
        or_fft2(P, cr, ci, -1);
        for (size_t q = 0; q < PP; ++q) {
            double a = cr[q] * kr[q] - ci[q] * ki[q];
            double b = cr[q] * ki[q] + ci[q] * kr[q];
            cr[q] = a;
            ci[q] = b;
        }
        or_fft2(P, cr, ci, +1);
        double inv = 1.0 / (double)PP;
        for (int64_t y = 0; y < G; ++y)
            for (int64_t x = 0; x < G; ++x)
                out[(size_t)c * G * G + y * G + x] = cr[y * P + x] * inv;
    }
    free(kr); free(ki); free(cr); free(ci);
    return 0;
}

/* Same interaction by the direct O(G^4) sum (small G; pins the FFT route). */
void or_conv_grid_direct(int64_t G, double s, double gamma, int nch, const double* in,
                         double* out) {
    for (int c = 0; c < nch; ++c)
        for (int64_t py = 0; py < G; ++py)
            for (int64_t px = 0; px < G; ++px) {
                double acc = 0.0;
                for (int64_t qy = 0; qy < G; ++qy)
                    for (int64_t qx = 0; qx < G; ++qx) {
                        double dx = (double)(px - qx) * s, dy = (double)(py - qy) * s;
                        acc += or_kernel(dx * dx + dy * dy, gamma) *
                               in[(size_t)c * G * G + qy * G + qx];
                    }
                out[(size_t)c * G * G + py * G + px] = acc;
            }
}

/* ------------------------------------------------------------------------- */
/* ibFFT repulsion, Sec. 3.4, in the paper's three-sum form (Eq. Fr1/Fr2 with */
/* v_j = 1, x_j, y_j of Eq. kernelproduct).                                   */
/*  grid: lo (origin of both axes), h (box side), n_int boxes per axis, k.    */
/*  Grid node (a, l) of an axis sits at lo + (a + (l + 1/2)/k) h  (reading:   */
/*  k interior equispaced nodes per box, spacing h/k across box borders).     */
/*  xyf: FP32 positions used for the box decision only.                       */
/* ------------------------------------------------------------------------- */
int or_rep_fft(int64_t n, const double* xy, const float* xyf, const double* wr, double gamma, int k,
               double lo, double h, int n_int, int64_t P, double* frep /* 2n */) {
    int64_t G = (int64_t)n_int * k;
    size_t GG = (size_t)G * (size_t)G;
    double* ch = (double*)calloc(3 * GG, sizeof(double));   /* C_1, C_x, C_y */
    double* psi = (double*)malloc(3 * GG * sizeof(double)); /* Psi_1, Psi_x, Psi_y */
    int* box = (int*)malloc(sizeof(int) * 2 * (size_t)(n > 0 ? n : 1));
    double* wts = (double*)malloc(sizeof(double) * 2 * (size_t)k * (size_t)(n > 0 ? n : 1));
    if (!ch || !psi || !box || !wts) { free(ch); free(psi); free(box); free(wts); return -2; }
    float lof = (float)lo, hf = (float)h;
    /* Step 1: projection onto the grid (Lagrange weights, per box). */
    for (int64_t i = 0; i < n; ++i) {
        for (int ax = 0; ax < 2; ++ax) {
            int a = or_box_f32(xyf[2 * i + ax], lof, hf, n_int);
            double u = (xy[2 * i + ax] - lo) / h - (double)a;
            box[2 * i + ax] = a;
            or_lagrange(k, u, wts + (2 * i + ax) * k);
        }
        const double* wx = wts + (2 * i) * k;
        const double* wy = wts + (2 * i + 1) * k;
        for (int ly = 0; ly < k; ++ly)
            for (int lx = 0; lx < k; ++lx) {
                int64_t qy = (int64_t)box[2 * i + 1] * k + ly, qx = (int64_t)box[2 * i] * k + lx;
                double w = or_w(wr, i) * wx[lx] * wy[ly];  /* charge r_i per node */
                size_t q = (size_t)qy * G + qx;
                ch[q] += w;
                ch[GG + q] += w * xy[2 * i];
                ch[2 * GG + q] += w * xy[2 * i + 1];
            }
    }
    /* Step 2: interaction of the grid nodes (spacing h/k) by FFT. */
    int rc = or_conv_grid_fft(G, P, h / k, gamma, 3, ch, psi);
    if (rc != 0) { free(ch); free(psi); free(box); free(wts); return rc; }
    /* Step 3: back-projection and Eq. (Fr1)/(Fr2). */
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        const double* wx = wts + (2 * i) * k;
        const double* wy = wts + (2 * i + 1) * k;
        double p1 = 0.0, px = 0.0, py = 0.0;
        for (int ly = 0; ly < k; ++ly)
            for (int lx = 0; lx < k; ++lx) {
                int64_t qy = (int64_t)box[2 * i + 1] * k + ly, qx = (int64_t)box[2 * i] * k + lx;
                double w = wx[lx] * wy[ly];
                size_t q = (size_t)qy * G + qx;
                p1 += w * psi[q];
                px += w * psi[GG + q];
                py += w * psi[2 * GG + q];
            }
        frep[2 * i] = or_w(wr, i) * (xy[2 * i] * p1 - px);
        frep[2 * i + 1] = or_w(wr, i) * (xy[2 * i + 1] * p1 - py);
    }
    free(ch); free(psi); free(box); free(wts);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Position update. The paper only says the resultant force moves each node   */
/* until convergence (Sec. 3.1) and implies 300 iterations (Sec. 4.1); the    */
/* schedule is a reading: a step capped at s_t along D(i), with s_t cooled    */
/* geometrically from s0 to s_min over T iterations.                          */
/* ------------------------------------------------------------------------- */
double or_step_size(int64_t t, int64_t T, double s0, double smin) {
    if (T <= 1) return s0;
    if (t > T - 1) t = T - 1;
    return s0 * pow(smin / s0, (double)t / (double)(T - 1));
}

void or_update(int64_t n, double* xy, const double* D, double s) {
    for (int64_t i = 0; i < n; ++i) {
        double dx = D[2 * i], dy = D[2 * i + 1];
        double norm = sqrt(dx * dx + dy * dy);
        double c = (norm > s) ? s / norm : 1.0;
        xy[2 * i] += c * dx;
        xy[2 * i + 1] += c * dy;
    }
}

/* ------------------------------------------------------------------------- */
/* Iteration driver: `iters` synchronous iterations starting at t0.           */
/* mode 0: exact repulsion; mode 1: ibFFT repulsion with (k, n_int_min,       */
/* grid_max, policy, P); P = 0 picks the smallest power of two >= 2G - 1.     */
/* ------------------------------------------------------------------------- */
static int64_t or_nextpow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

/* k of iteration t of a T-iteration run (Sec. 3.4 "Choices of k"). k > 0 is fixed;
 * k = 0 is the paper's dynamic strategy: 1 while t < floor(0.9 T), 2 while
 * t < floor(0.95 T), then 3 (also for t >= T). With T = 300 that is 270 iterations at
 * k = 1, the count Sec. 4.2 mentions. */
int or_k_of_iter(int k, int64_t t, int64_t T) {
    if (k > 0) return k;
    if (t < (9 * T) / 10) return 1;
    if (t < (19 * T) / 20) return 2;
    return 3;
}

int or_iterate(int64_t n, int64_t m, const int32_t* edges, double* xy, const double* wr,
               const double* wa, double alpha, double beta, double gamma, int mode, int k,
               int n_int_min, int grid_max, int policy, int64_t P, double s0, double smin, int64_t T,
               int64_t t0, int64_t iters) {
    double* frep = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    double* fatt = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    float* xyf = (float*)malloc(sizeof(float) * 2 * (size_t)(n > 0 ? n : 1));
    if (!frep || !fatt || !xyf) { free(frep); free(fatt); free(xyf); return -2; }
    int rc = 0;
    for (int64_t t = t0; t < t0 + iters && rc == 0; ++t) {
        if (mode == 0) {
            or_rep_exact(n, xy, wr, gamma, 0, n, frep);
        } else {
            for (int64_t i = 0; i < 2 * n; ++i) xyf[i] = (float)xy[i];
            const int kt = or_k_of_iter(k, t, T);
            /* Under the dynamic strategy N_int has one cap for every k, floor(grid_max / 3):
             * the paper's N_int rule (Sec. 3.4 "Choices of k") does not depend on k, so the
             * k = 1 grid is a third of the k = 3 grid per axis (reading R9b). */
            const int gm = (k == 0) ? kt * (grid_max / 3) : grid_max;
            double g[5];
            or_grid_policy(n, xyf, kt, n_int_min, gm, policy, g);
            int n_int = (int)g[2];
            int64_t PP = P > 0 ? P : or_nextpow2(2 * (int64_t)n_int * kt - 1);
            rc = or_rep_fft(n, xy, xyf, wr, gamma, kt, g[0], g[1], n_int, PP, frep);
        }
        or_att(n, m, edges, xy, wa, alpha, beta, fatt);
        for (int64_t i = 0; i < 2 * n; ++i) frep[i] += fatt[i];
        or_update(n, xy, frep, or_step_size(t, T, s0, smin));
    }
    free(frep); free(fatt); free(xyf);
    return rc;
}
