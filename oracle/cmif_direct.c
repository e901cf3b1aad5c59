/*
 * CPU oracle for the cross-mutual information function (CMIF).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and it never calls it.
 *
 * What it computes is the plain definition, the paper's *direct method*
 * (Sec. 2.2): for every displacement chi, walk the overlap of A and the
 * shifted B, increment the joint histogram bin (a, b), the marginal bins a
 * and b, and the overlap count N wherever both masks are 1, then form the
 * entropies in FP64 from relative frequencies (Eq. margentropy,
 * Eq. jointentropy, Eq. finalentropy) and MI = H_A + H_B - H_AB
 * (Eq. mientropy).  Conventions of Sec. 3.2: 0/0 = 0 and 0 log 0 = 0, so a
 * shift with N = 0 has MI = 0.
 *
 * Shift convention (Eq. cc, Eq. cmif): T_chi[B](x) = B(x + chi), so the
 * counts at chi pair A(y, x) with B(y + dy, x + dx).  The full linear range
 * is dy in [-(H_A-1), H_B-1], dx in [-(W_A-1), W_B-1]; the map index of
 * (dy, dx) is (dy + H_A - 1) * (W_A + W_B - 1) + (dx + W_A - 1).
 *
 * Labels under a mask value 1 must lie in [0, K); anything else is an
 * error (ORACLE_ERR_LABEL_RANGE).  Labels under mask 0 are ignored.  A NULL
 * mask means all ones.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_LABEL_RANGE 2
#define ORACLE_ERR_INTERNAL 3

static int labels_in_range(const int32_t *X, const uint8_t *M, long n, int K)
{
    for (long i = 0; i < n; ++i) {
        if (M && !M[i]) continue;
        if (X[i] < 0 || X[i] >= K) return 0;
    }
    return 1;
}

/* Histograms of the overlap at one displacement, by a direct walk (Sec. 2.2). */
static int direct_counts(const int32_t *A, const uint8_t *MA, int HA, int WA,
                         const int32_t *B, const uint8_t *MB, int HB, int WB,
                         int KA, int KB, int dy, int dx,
                         int64_t *J, int64_t *CA, int64_t *CB, int64_t *N)
{
    memset(J, 0, sizeof(int64_t) * (size_t)KA * KB);
    memset(CA, 0, sizeof(int64_t) * (size_t)KA);
    memset(CB, 0, sizeof(int64_t) * (size_t)KB);
    int64_t n = 0;
    int y0 = dy < 0 ? -dy : 0, y1 = HA < HB - dy ? HA : HB - dy;
    int x0 = dx < 0 ? -dx : 0, x1 = WA < WB - dx ? WA : WB - dx;
    for (int y = y0; y < y1; ++y) {
        const int32_t *ar = A + (size_t)y * WA;
        const int32_t *br = B + (size_t)(y + dy) * WB + dx;
        const uint8_t *mar = MA ? MA + (size_t)y * WA : NULL;
        const uint8_t *mbr = MB ? MB + (size_t)(y + dy) * WB + dx : NULL;
        for (int x = x0; x < x1; ++x) {
            if (mar && !mar[x]) continue;
            if (mbr && !mbr[x]) continue;
            int a = ar[x], b = br[x];
            J[(size_t)a * KB + b] += 1;
            CA[a] += 1;
            CB[b] += 1;
            n += 1;
        }
    }
    *N = n;
    /* The marginals must be the row / column sums of the joint (Eq. number). */
    for (int a = 0; a < KA; ++a) {
        int64_t s = 0;
        for (int b = 0; b < KB; ++b) s += J[(size_t)a * KB + b];
        if (s != CA[a]) return ORACLE_ERR_INTERNAL;
    }
    for (int b = 0; b < KB; ++b) {
        int64_t s = 0;
        for (int a = 0; a < KA; ++a) s += J[(size_t)a * KB + b];
        if (s != CB[b]) return ORACLE_ERR_INTERNAL;
    }
    return ORACLE_OK;
}

/* -p log2 p with p = c / n; 0 log 0 = 0 (Sec. 3.2). */
static double neg_plogp(int64_t c, int64_t n)
{
    if (c == 0) return 0.0;
    double p = (double)c / (double)n;
    return -p * log2(p);
}

/* Entropies of Eq. finalentropy, term by term, and MI by Eq. mientropy. */
static double mi_from_counts(const int64_t *J, const int64_t *CA, const int64_t *CB,
                             int64_t N, int KA, int KB, double *hA, double *hB, double *hAB)
{
    double HA = 0, HB = 0, HAB = 0;
    if (N > 0) {
        for (int a = 0; a < KA; ++a) HA += neg_plogp(CA[a], N);
        for (int b = 0; b < KB; ++b) HB += neg_plogp(CB[b], N);
        for (int a = 0; a < KA; ++a)
            for (int b = 0; b < KB; ++b) HAB += neg_plogp(J[(size_t)a * KB + b], N);
    }
    if (hA) *hA = HA;
    if (hB) *hB = HB;
    if (hAB) *hAB = HAB;
    return HA + HB - HAB;
}

static int check_args(const int32_t *A, int HA, int WA, const int32_t *B, int HB, int WB, int KA, int KB)
{
    if (!A || !B || HA <= 0 || WA <= 0 || HB <= 0 || WB <= 0 || KA <= 0 || KB <= 0) return ORACLE_ERR_ARG;
    return ORACLE_OK;
}

/*
 * Full CMIF map over the linear shift range.  Outputs (row-major over
 * (dy, dx) as described above, R = H_A+H_B-1 rows, C = W_A+W_B-1 cols):
 *   mi[R*C]            MI in bits (FP64)
 *   n[R*C]             overlap count N (nullable)
 *   joint[KA*KB][R*C]  joint counts C_AB^{a,b} (nullable)
 *   marg_a[KA][R*C]    C_A^a (nullable), marg_b[KB][R*C] C_B^b (nullable)
 *   ent[3][R*C]        H_A, H_B, H_AB (nullable)
 */
int oracle_cmif(const int32_t *A, const uint8_t *MA, int HA, int WA,
                const int32_t *B, const uint8_t *MB, int HB, int WB,
                int KA, int KB, double *mi, int64_t *n, int32_t *joint,
                int32_t *marg_a, int32_t *marg_b, double *ent, int nthreads)
{
    int st = check_args(A, HA, WA, B, HB, WB, KA, KB);
    if (st) return st;
    if (!mi) return ORACLE_ERR_ARG;
    if (!labels_in_range(A, MA, (long)HA * WA, KA) || !labels_in_range(B, MB, (long)HB * WB, KB))
        return ORACLE_ERR_LABEL_RANGE;
    const int R = HA + HB - 1, C = WA + WB - 1;
    const long RC = (long)R * C;
    int err = ORACLE_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(|:err)
#endif
    {
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)KA * KB);
        int64_t *CA = (int64_t *)malloc(sizeof(int64_t) * (size_t)KA);
        int64_t *CB = (int64_t *)malloc(sizeof(int64_t) * (size_t)KB);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int r = 0; r < R; ++r) {
            int dy = r - (HA - 1);
            for (int c = 0; c < C; ++c) {
                int dx = c - (WA - 1);
                int64_t N;
                long o = (long)r * C + c;
                if (direct_counts(A, MA, HA, WA, B, MB, HB, WB, KA, KB, dy, dx, J, CA, CB, &N)) err = ORACLE_ERR_INTERNAL;
                double h[3];
                mi[o] = mi_from_counts(J, CA, CB, N, KA, KB, &h[0], &h[1], &h[2]);
                if (n) n[o] = N;
                if (ent) { ent[o] = h[0]; ent[RC + o] = h[1]; ent[2 * RC + o] = h[2]; }
                if (joint)
                    for (int p = 0; p < KA * KB; ++p) joint[(long)p * RC + o] = (int32_t)J[p];
                if (marg_a)
                    for (int a = 0; a < KA; ++a) marg_a[(long)a * RC + o] = (int32_t)CA[a];
                if (marg_b)
                    for (int b = 0; b < KB; ++b) marg_b[(long)b * RC + o] = (int32_t)CB[b];
            }
        }
        free(J); free(CA); free(CB);
    }
    return err;
}

/*
 * CMIF at a list of displacements (dy[i], dx[i]), for sampled checks of
 * large maps.  joint (nullable) is [n_shifts][KA*KB].
 */
int oracle_cmif_at(const int32_t *A, const uint8_t *MA, int HA, int WA,
                   const int32_t *B, const uint8_t *MB, int HB, int WB,
                   int KA, int KB, int n_shifts, const int32_t *dys, const int32_t *dxs,
                   double *mi, int64_t *n, int32_t *joint, double *ent, int nthreads)
{
    int st = check_args(A, HA, WA, B, HB, WB, KA, KB);
    if (st) return st;
    if (!mi || !dys || !dxs || n_shifts < 0) return ORACLE_ERR_ARG;
    if (!labels_in_range(A, MA, (long)HA * WA, KA) || !labels_in_range(B, MB, (long)HB * WB, KB))
        return ORACLE_ERR_LABEL_RANGE;
    for (int i = 0; i < n_shifts; ++i)
        if (dys[i] < -(HA - 1) || dys[i] > HB - 1 || dxs[i] < -(WA - 1) || dxs[i] > WB - 1) return ORACLE_ERR_ARG;
    int err = ORACLE_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(|:err)
#endif
    {
        int64_t *J = (int64_t *)malloc(sizeof(int64_t) * (size_t)KA * KB);
        int64_t *CA = (int64_t *)malloc(sizeof(int64_t) * (size_t)KA);
        int64_t *CB = (int64_t *)malloc(sizeof(int64_t) * (size_t)KB);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int i = 0; i < n_shifts; ++i) {
            int64_t N;
            if (direct_counts(A, MA, HA, WA, B, MB, HB, WB, KA, KB, dys[i], dxs[i], J, CA, CB, &N)) err = ORACLE_ERR_INTERNAL;
            double h[3];
            mi[i] = mi_from_counts(J, CA, CB, N, KA, KB, &h[0], &h[1], &h[2]);
            if (n) n[i] = N;
            if (ent) { ent[3 * i] = h[0]; ent[3 * i + 1] = h[1]; ent[3 * i + 2] = h[2]; }
            if (joint)
                for (int p = 0; p < KA * KB; ++p) joint[(long)i * KA * KB + p] = (int32_t)J[p];
        }
        free(J); free(CA); free(CB);
    }
    return err;
}

/*
 * Nearest-neighbour rotation of the floating image (Sec. 3.6: B is warped
 * with NN interpolation because its labels are categorical).  The paper does
 * not fix the centre, canvas or sign; the reading used here: centre
 * c = ((H-1)/2, (W-1)/2) in (row, col), canvas = B's own size, and the output
 * pixel (i, j) takes the source
 *     col_s = c_col + u cos(theta) - v sin(theta)
 *     row_s = c_row + u sin(theta) + v cos(theta),  u = j - c_col, v = i - c_row,
 * each rounded half away from zero.  (That is, the image content turns by
 * theta counter-clockwise on screen, rows pointing down.)  The output mask is
 * 1 iff the source lies inside B and M_B(source) = 1; elsewhere label and
 * mask are 0.
 */
int oracle_warp_nn(const int32_t *B, const uint8_t *MB, int H, int W, double theta,
                   int32_t *outB, uint8_t *outM)
{
    if (!B || !outB || !outM || H <= 0 || W <= 0) return ORACLE_ERR_ARG;
    const double cr = (H - 1) * 0.5, cc = (W - 1) * 0.5;
    const double ct = cos(theta), sn = sin(theta);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double u = j - cc, v = i - cr;
            double xs = cc + u * ct - v * sn;
            double ys = cr + u * sn + v * ct;
            long si = lround(ys), sj = lround(xs);
            long o = (long)i * W + j;
            if (si >= 0 && si < H && sj >= 0 && sj < W && (!MB || MB[si * W + sj])) {
                outB[o] = B[si * W + sj];
                outM[o] = 1;
            } else {
                outB[o] = 0;
                outM[o] = 0;
            }
        }
    return ORACLE_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
