/*
 * Numeric oracle for the DAG-node kernels (test infrastructure only).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It shares no code with the CUDA path.
 *
 * Every routine is the plain definition of what one node computes, in fp64,
 * one element after the other, in the order the definition is written.
 * Inputs arrive as fp64 copies of the fp32 (or int32) device inputs.
 *
 * The paper (Section IV-B, "Benchmark Suite") names the six benchmarks
 * (VEC, B&S, IMG, ML, HITS, DL) but prints no formulas or kernels; where the
 * text is silent, the reading taken is stated beside the routine.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared numeric.c -lm
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

/* ------------------------------------------------------------------ VEC --
 * Section IV-B, VEC: "the sum of differences of 2 squared vectors".
 * K1: x := x*x, K2: y := y*y, K3: z = sum_i (x_i - y_i) over the squared
 * arrays (program order: K3 runs after K1 and K2).                        */
void orc_square(const double *x, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = x[i] * x[i];
}

double orc_sum_diff(const double *x, const double *y, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += x[i] - y[i];
    return s;
}

/* Sum of |x_i - y_i|: the condition scale of orc_sum_diff.               */
double orc_sum_abs_diff(const double *x, const double *y, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += fabs(x[i] - y[i]);
    return s;
}

/* ------------------------------------------------------------------ B&S --
 * Section IV-B, B&S: Black-Scholes price of a European call.
 *   d1 = (ln(S/K) + (r + sigma^2/2) T) / (sigma sqrt(T))
 *   d2 = d1 - sigma sqrt(T)
 *   C  = S N(d1) - K exp(-r T) N(d2)
 * with N the standard normal CDF, N(x) = erfc(-x / sqrt(2)) / 2 (exact
 * erfc from libm, not a polynomial approximation).                        */
double orc_cnd(double x)
{
    return 0.5 * erfc(-x / sqrt(2.0));
}

void orc_bs_call(const double *S, double *C, int64_t n,
                 double K, double r, double sigma, double T)
{
    for (int64_t i = 0; i < n; ++i) {
        double d1 = (log(S[i] / K) + (r + 0.5 * sigma * sigma) * T)
                    / (sigma * sqrt(T));
        double d2 = d1 - sigma * sqrt(T);
        C[i] = S[i] * orc_cnd(d1) - K * exp(-r * T) * orc_cnd(d2);
    }
}

/* Magnitude of the two terms of C, S N(d1) + K exp(-rT) N(d2): the
 * condition scale of the difference (C is small where they nearly cancel). */
void orc_bs_call_scale(const double *S, double *A, int64_t n,
                       double K, double r, double sigma, double T)
{
    for (int64_t i = 0; i < n; ++i) {
        double d1 = (log(S[i] / K) + (r + 0.5 * sigma * sigma) * T)
                    / (sigma * sqrt(T));
        double d2 = d1 - sigma * sqrt(T);
        A[i] = S[i] * orc_cnd(d1) + K * exp(-r * T) * orc_cnd(d2);
    }
}

/* ------------------------------------------------------------------ IMG --
 * Section IV-B, IMG: a sharpened picture combined with copies blurred at low
 * and medium frequency.  Readings (the paper gives no formulas):
 *   Gaussian blur of radius R with weights w_k = exp(-k^2/(2 sigma^2)),
 *   k = -R..R, normalised to sum 1; 5x5 is R=2, sigma=1; 9x9 is R=4,
 *   sigma=2.  Pixels outside the image take the value of the nearest edge
 *   pixel (clamp-to-edge).  Images are row-major, rows x cols.            */
static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

void orc_gauss_weights(int R, double sigma, double *w)
{
    double s = 0.0;
    for (int k = -R; k <= R; ++k) {
        w[k + R] = exp(-(double)(k * k) / (2.0 * sigma * sigma));
        s += w[k + R];
    }
    for (int k = 0; k < 2 * R + 1; ++k)
        w[k] /= s;
}

/* out[r][c] = sum_{i,j=-R..R} w[i] w[j] img[clamp(r+i)][clamp(c+j)]:
 * the 2-D definition of the separable blur, evaluated directly.           */
void orc_blur(const double *img, double *out, int64_t rows, int64_t cols,
              const double *w, int R)
{
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            double s = 0.0;
            for (int i = -R; i <= R; ++i) {
                int64_t rr = clampi(r + i, 0, rows - 1);
                for (int j = -R; j <= R; ++j) {
                    int64_t cc = clampi(c + j, 0, cols - 1);
                    s += w[i + R] * w[j + R] * img[rr * cols + cc];
                }
            }
            out[r * cols + c] = s;
        }
}

/* Sobel gradient magnitude, clamp-to-edge:
 *   gx = sum_{i,j} Kx[i][j] in[r+i][c+j], Kx = [[-1,0,1],[-2,0,2],[-1,0,1]]
 *   gy = sum_{i,j} Ky[i][j] in[r+i][c+j], Ky = Kx transposed
 *   out = sqrt(gx^2 + gy^2)                                              */
void orc_sobel(const double *in, double *out, int64_t rows, int64_t cols)
{
    static const double Kx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            double gx = 0.0, gy = 0.0;
            for (int i = -1; i <= 1; ++i)
                for (int j = -1; j <= 1; ++j) {
                    double v = in[clampi(r + i, 0, rows - 1) * cols
                                  + clampi(c + j, 0, cols - 1)];
                    gx += Kx[i + 1][j + 1] * v;
                    gy += Kx[j + 1][i + 1] * v;
                }
            out[r * cols + c] = sqrt(gx * gx + gy * gy);
        }
}

/* Condition scale of the Sobel magnitude at each pixel: the sum of the
 * absolute values of the terms of both gradients, sum |Kx v| + sum |Ky v|
 * over the clamped 3x3 window.  A rounding error of a few units in the last
 * place of each term bounds the error of gx and gy, and so of
 * sqrt(gx^2 + gy^2), by a small multiple of this scale (the reading used for
 * every sum of terms of mixed sign).                                      */
void orc_sobel_scale(const double *in, double *out, int64_t rows, int64_t cols)
{
    static const double Kx[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c) {
            double sx = 0.0, sy = 0.0;
            for (int i = -1; i <= 1; ++i)
                for (int j = -1; j <= 1; ++j) {
                    double v = in[clampi(r + i, 0, rows - 1) * cols
                                  + clampi(c + j, 0, cols - 1)];
                    sx += fabs(Kx[i + 1][j + 1] * v);
                    sy += fabs(Kx[j + 1][i + 1] * v);
                }
            out[r * cols + c] = sx + sy;
        }
}

void orc_minmax(const double *x, int64_t n, double *mn, double *mx)
{
    double lo = x[0], hi = x[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < lo) lo = x[i];
        if (x[i] > hi) hi = x[i];
    }
    *mn = lo;
    *mx = hi;
}

/* Linear contrast stretch to [0, 1]; a flat image (max == min) maps to 0. */
void orc_extend(const double *in, double mn, double mx, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = (mx > mn) ? (in[i] - mn) / (mx - mn) : 0.0;
}

/* Unsharp mask: S = img + alpha (img - blur).                            */
void orc_unsharp(const double *img, const double *blur, double alpha,
                 double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = img[i] + alpha * (img[i] - blur[i]);
}

/* Combine: the sharpened image where the fine-scale edge mask e5 is high,
 * else the low-blur copy where the coarse mask e9 is high, else the
 * high-blur copy:  out = e5 S + (1 - e5) (e9 b5 + (1 - e9) b9).           */
void orc_combine(const double *S, const double *b5, const double *b9,
                 const double *e5, const double *e9, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = e5[i] * S[i]
                 + (1.0 - e5[i]) * (e9[i] * b5[i] + (1.0 - e9[i]) * b9[i]);
}

/* ------------------------------------------------------------------- ML --
 * Section IV-B, ML: naive-Bayes and ridge-regression classifiers combined by
 * a softmax of each and the average of the scores.  Both score nodes are
 *   S[i][c] = bias[c] + sum_f X[i][f] T[f][c]
 * (multinomial naive Bayes with a log-probability table T and log prior
 * bias; ridge with weights T and intercept bias).  X is row-major rows x
 * feats, T row-major feats x classes.                                     */
void orc_scores(const double *X, int64_t rows, int64_t feats,
                const double *T, int64_t classes, const double *bias,
                double *S)
{
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t c = 0; c < classes; ++c) {
            double s = bias[c];
            for (int64_t f = 0; f < feats; ++f)
                s += X[i * feats + f] * T[f * classes + c];
            S[i * classes + c] = s;
        }
}

/* Sum over f of |X[i][f] T[f][c]| + |bias[c]|: condition scale per output. */
void orc_scores_abs(const double *X, int64_t rows, int64_t feats,
                    const double *T, int64_t classes, const double *bias,
                    double *A)
{
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t c = 0; c < classes; ++c) {
            double s = fabs(bias[c]);
            for (int64_t f = 0; f < feats; ++f)
                s += fabs(X[i * feats + f] * T[f * classes + c]);
            A[i * classes + c] = s;
        }
}

/* Row softmax: P[i][c] = exp(S[i][c] - m_i) / sum_k exp(S[i][k] - m_i),
 * m_i = max_k S[i][k].                                                   */
void orc_softmax_rows(const double *S, double *P, int64_t rows,
                      int64_t classes)
{
    for (int64_t i = 0; i < rows; ++i) {
        double m = S[i * classes];
        for (int64_t c = 1; c < classes; ++c)
            if (S[i * classes + c] > m) m = S[i * classes + c];
        double z = 0.0;
        for (int64_t c = 0; c < classes; ++c)
            z += exp(S[i * classes + c] - m);
        for (int64_t c = 0; c < classes; ++c)
            P[i * classes + c] = exp(S[i * classes + c] - m) / z;
    }
}

/* label_i = argmax_c (P1[i][c] + P2[i][c]); ties go to the lowest c.
 * margin_i = best - second best (0 when tied): rows whose margin is below
 * the comparison tolerance accept either label.                         */
void orc_argmax_sum(const double *P1, const double *P2, int64_t rows,
                    int64_t classes, int32_t *labels, double *margin)
{
    for (int64_t i = 0; i < rows; ++i) {
        int64_t best = 0;
        double bv = P1[i * classes] + P2[i * classes];
        double second = -INFINITY;
        for (int64_t c = 1; c < classes; ++c) {
            double v = P1[i * classes + c] + P2[i * classes + c];
            if (v > bv) {
                second = bv;
                bv = v;
                best = c;
            } else if (v > second) {
                second = v;
            }
        }
        labels[i] = (int32_t)best;
        margin[i] = (classes > 1) ? bv - second : INFINITY;
    }
}

/* ----------------------------------------------------------------- HITS --
 * Section IV-B, HITS (Kleinberg's hubs and authorities) with sparse
 * matrix-vector products on the adjacency matrix and its transpose.
 * CSR: row i holds the nonzeros col[rowptr[i] .. rowptr[i+1]).
 *   y_i = sum_{k in row i} val_k x_{col_k}                                 */
void orc_spmv_csr(int64_t nrows, const int64_t *rowptr, const int32_t *col,
                  const double *val, const double *x, double *y)
{
    for (int64_t i = 0; i < nrows; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s += val[k] * x[col[k]];
        y[i] = s;
    }
}

/* Row sums of |val_k x_col_k|: condition scale of each y_i.              */
void orc_spmv_csr_abs(int64_t nrows, const int64_t *rowptr,
                      const int32_t *col, const double *val, const double *x,
                      double *y)
{
    for (int64_t i = 0; i < nrows; ++i) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            s += fabs(val[k] * x[col[k]]);
        y[i] = s;
    }
}

double orc_l2norm(const double *x, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += x[i] * x[i];
    return sqrt(s);
}

/* x := x / nrm; a zero norm leaves x unscaled.                           */
void orc_scale(const double *x, double nrm, double *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = (nrm > 0.0) ? x[i] / nrm : x[i];
}

/* ------------------------------------------------------------------- DL --
 * Section IV-B, DL: a convolutional network projects two images to
 * low-dimensional embeddings and combines them with a dense layer.
 * Readings (the paper gives no layer sizes): per branch a 3x3 convolution
 * with 3 input and C output channels, zero padding 1, stride 1, plus bias,
 * ReLU, and 2x2 max-pooling with stride 2; NCHW layout.                    */
void orc_conv3x3_relu_pool(const double *x, int64_t n, int64_t cin, int64_t h,
                           int64_t w, const double *wt, const double *bias,
                           int64_t cout, double *out)
{
    const int64_t ho = h / 2, wo = w / 2;
    for (int64_t b = 0; b < n; ++b)
        for (int64_t co = 0; co < cout; ++co)
            for (int64_t py = 0; py < ho; ++py)
                for (int64_t px = 0; px < wo; ++px) {
                    double best = -INFINITY;
                    for (int64_t sy = 0; sy < 2; ++sy)
                        for (int64_t sx = 0; sx < 2; ++sx) {
                            const int64_t y = 2 * py + sy, xx = 2 * px + sx;
                            double s = bias[co];
                            for (int64_t ci = 0; ci < cin; ++ci)
                                for (int64_t dy = -1; dy <= 1; ++dy)
                                    for (int64_t dx = -1; dx <= 1; ++dx) {
                                        const int64_t yy = y + dy, xq = xx + dx;
                                        if (yy < 0 || yy >= h || xq < 0 || xq >= w) continue;
                                        s += wt[((co * cin + ci) * 3 + (dy + 1)) * 3 + (dx + 1)]
                                             * x[((b * cin + ci) * h + yy) * w + xq];
                                    }
                            const double r = s > 0.0 ? s : 0.0;
                            if (r > best) best = r;
                        }
                    out[((b * cout + co) * ho + py) * wo + px] = best;
                }
}

/* Global average pool: e[p] = mean over the hw values of plane p.         */
void orc_avgpool(const double *x, int64_t planes, int64_t hw, double *e)
{
    for (int64_t p = 0; p < planes; ++p) {
        double s = 0.0;
        for (int64_t i = 0; i < hw; ++i)
            s += x[p * hw + i];
        e[p] = s / (double)hw;
    }
}

/* Concatenate two n x c embeddings to n x 2c and apply a dense layer:
 * out[b][j] = bias[j] + sum_i cat[b][i] wd[i][j], wd row-major 2c x classes. */
void orc_concat_dense(const double *e1, const double *e2, int64_t n, int64_t c,
                      const double *wd, const double *bias, int64_t classes,
                      double *out)
{
    for (int64_t b = 0; b < n; ++b)
        for (int64_t j = 0; j < classes; ++j) {
            double s = bias[j];
            for (int64_t i = 0; i < c; ++i)
                s += e1[b * c + i] * wd[i * classes + j];
            for (int64_t i = 0; i < c; ++i)
                s += e2[b * c + i] * wd[(c + i) * classes + j];
            out[b * classes + j] = s;
        }
}
