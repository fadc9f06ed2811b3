/*
 * CPU oracle for the tenant kernels: test infrastructure only.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library. It shares no code with the GPU path (no header, no
 * helper, no constant table): every function here is the plain definition of
 * what the tenant computes, written out in the obvious loop order.
 *
 * The paper's eight benchmark kernels (Section 5.1, Table 4) come from suites
 * that are not available; the tenant set below follows the synthetic mix the
 * scheduling experiments need (the co-scheduling method of Section 4 is
 * independent of what a tenant computes, it only needs independent thread
 * blocks, Section 2.2 assumption 2). Four of the paper's kernels are written
 * here from their textbook definitions: TEA, SAD, the 7-point stencil and
 * MRI-Q (which adds a sine/cosine recipe, below).
 *
 * Floating point: every float operation is a separately rounded IEEE binary32
 * operation; fused multiply-add appears only where fmaf() is written. Build
 * with -ffp-contract=off and without -ffast-math.
 *
 * Black-Scholes uses two transcendental functions written from published
 * methods (no C library exp/log on that path, so that a GPU implementation
 * of the same written recipe can be compared bit for bit):
 *   or_expf: Cody-Waite argument reduction x = n*ln2 + r with a two-part ln2
 *            (W. J. Cody, W. Waite, "Software Manual for the Elementary
 *            Functions", 1980), then the degree-7 Taylor polynomial of e^r in
 *            Horner form with fmaf, then scaling by 2^n through exponent bits.
 *   or_logf: x = 2^e * m with m in [sqrt(1/2), sqrt(2)), log m = 2 atanh(t),
 *            t = (m-1)/(m+1), odd series to t^9 (Horner in t^2 with fmaf),
 *            plus e*ln2 in two parts.
 *   CND:     Abramowitz & Stegun 26.2.17 (|error| < 7.5e-8) with reflection.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ exp / log */

static float f_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_from_f(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

float or_expf(float x) {
    if (x != x) return x;
    if (x > 88.7228394f) return INFINITY;
    if (x < -103.972694f) return 0.0f;
    const float log2e = 1.44269504f;
    const float ln2_hi = 0.693145751953125f;      /* ln 2 with 9 low bits cleared */
    const float ln2_lo = 1.42860677e-06f;         /* ln 2 - ln2_hi */
    float t = x * log2e;
    float n = rintf(t);
    float r = fmaf(-n, ln2_hi, x);
    r = fmaf(-n, ln2_lo, r);
    /* e^r = sum_{k=0..7} r^k / k!  (Horner, innermost first) */
    float p = 1.98412698e-04f;                    /* 1/5040 */
    p = fmaf(p, r, 1.38888889e-03f);              /* 1/720 */
    p = fmaf(p, r, 8.33333333e-03f);              /* 1/120 */
    p = fmaf(p, r, 4.16666667e-02f);              /* 1/24 */
    p = fmaf(p, r, 1.66666667e-01f);              /* 1/6 */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int ni = (int)n;
    if (ni < -126) {                               /* subnormal result: two scalings */
        p = p * f_from_bits((uint32_t)(127 - 64) << 23);
        ni += 64;
    }
    if (ni > 127) {
        p = p * 2.0f;
        ni -= 1;
    }
    return p * f_from_bits((uint32_t)(ni + 127) << 23);
}

float or_logf(float x) {
    if (x != x) return x;
    if (x < 0.0f) return NAN;
    if (x == 0.0f) return -INFINITY;
    if (x == INFINITY) return x;
    int e_adj = 0;
    if (x < 1.17549435e-38f) {                     /* subnormal input */
        x = x * 16777216.0f;                       /* 2^24, exact */
        e_adj = -24;
    }
    uint32_t b = bits_from_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127 + e_adj;
    float m = f_from_bits((b & 0x007fffffu) | 0x3f800000u);  /* [1, 2) */
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    float num = m - 1.0f;
    float den = m + 1.0f;
    float t = num / den;
    float t2 = t * t;
    /* log m = 2t (1 + t^2/3 + t^4/5 + t^6/7 + t^8/9): the bracket minus one
       is s * t^2, added to the leading 2t with one fused operation */
    float s = 1.11111111e-01f;                     /* 1/9 */
    s = fmaf(s, t2, 1.42857143e-01f);              /* 1/7 */
    s = fmaf(s, t2, 2.00000000e-01f);              /* 1/5 */
    s = fmaf(s, t2, 3.33333333e-01f);              /* 1/3 */
    float st2 = s * t2;
    float tt = t + t;
    float lm = fmaf(tt, st2, tt);
    float fe = (float)e;
    float res = fmaf(fe, 1.42860677e-06f, lm);
    res = fmaf(fe, 0.693145751953125f, res);
    return res;
}

/* ------------------------------------------------------------ Black-Scholes */

static float or_cnd(float d) {
    const float a1 = 0.31938153f, a2 = -0.356563782f, a3 = 1.781477937f,
                a4 = -1.821255978f, a5 = 1.330274429f;
    float ad = fabsf(d);
    float pa = 0.2316419f * ad;
    float den = 1.0f + pa;
    float k = 1.0f / den;
    float poly = a5;
    poly = fmaf(poly, k, a4);
    poly = fmaf(poly, k, a3);
    poly = fmaf(poly, k, a2);
    poly = fmaf(poly, k, a1);
    poly = poly * k;
    float hd = 0.5f * d;
    float e = hd * d;
    float ex = or_expf(-e);
    float phi = 0.398942280f * ex;                 /* 1/sqrt(2 pi) */
    float c = phi * poly;                          /* 1 - N(|d|) */
    return (d > 0.0f) ? (1.0f - c) : c;
}

void or_blackscholes(const float* S, const float* K, const float* r, const float* v,
                     const float* T, float* call, float* put, int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
        float s = S[i], k = K[i], rr = r[i], vv = v[i], tt = T[i];
        float sqrtT = sqrtf(tt);
        float vsqrtT = vv * sqrtT;
        float q = s / k;
        float lq = or_logf(q);
        float h = 0.5f * vv;
        h = h * vv;
        float a = rr + h;
        a = a * tt;
        float num = lq + a;
        float d1 = num / vsqrtT;
        float d2 = d1 - vsqrtT;
        float c1 = or_cnd(d1);
        float c2 = or_cnd(d2);
        float m = rr * tt;
        float disc = or_expf(-m);
        float kd = k * disc;
        float t1 = s * c1;
        float t2 = kd * c2;
        call[i] = t1 - t2;
        float u2 = 1.0f - c2;
        float u1 = 1.0f - c1;
        float p1 = kd * u2;
        float p2 = s * u1;
        put[i] = p1 - p2;
    }
}

/* ------------------------------------------------------------ testing kernel (Section 4.3)
 * Thread g of nthreads: acc = 0; for round i < iters: for m < mem:
 * acc = acc + in[(g + (i mem + m) nthreads) mod n_in]; then alu times
 * acc = fmaf(acc, c1, c2); out[g] = acc. */

void or_testmix(const float* in, float* out, int64_t n_in, int64_t nthreads, int64_t iters, int64_t mem,
                int64_t alu, float c1, float c2) {
    for (int64_t g = 0; g < nthreads; ++g) {
        float acc = 0.0f;
        for (int64_t i = 0; i < iters; ++i) {
            for (int64_t m = 0; m < mem; ++m) acc = acc + in[(g + (i * mem + m) * nthreads) % n_in];
            for (int64_t q = 0; q < alu; ++q) acc = fmaf(acc, c1, c2);
        }
        out[g] = acc;
    }
}

/* ------------------------------------------------------------ gather */

void or_gather(const int32_t* a, const int32_t* idx, int32_t* out, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) out[i] = a[idx[i]];
}

/* ------------------------------------------------------------ FP32 GEMM
 * C[i][j] = fmaf chain over k = 0..K-1 ascending, starting from +0.0f. */

void or_gemm_f32(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K) {
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = 0; j < N; ++j) {
            float c = 0.0f;
            for (int64_t k = 0; k < K; ++k) c = fmaf(A[i * K + k], B[k * N + j], c);
            C[i * N + j] = c;
        }
}

/* one element (i,j) of the same definition, for sampled checks at full size */
void or_gemm_f32_sample(const float* A, const float* B, const int64_t* ii, const int64_t* jj,
                        float* out, int64_t ns, int64_t N, int64_t K) {
    for (int64_t s = 0; s < ns; ++s) {
        float c = 0.0f;
        for (int64_t k = 0; k < K; ++k) c = fmaf(A[ii[s] * K + k], B[k * N + jj[s]], c);
        out[s] = c;
    }
}

/* ------------------------------------------------------------ CSR SpMV
 * y32[r]: ascending fmaf chain from 0 (the definition in binary32);
 * y64[r]: the same sum in binary64 from exact products (reference value);
 * asum[r]: sum |val*x| in binary64 (scale for normwise error bounds). */

void or_spmv_csr(const int32_t* rowptr, const int32_t* col, const float* val, const float* x,
                 float* y32, double* y64, double* asum, int64_t nrows) {
    for (int64_t r = 0; r < nrows; ++r) {
        float acc = 0.0f;
        double a64 = 0.0, s64 = 0.0;
        for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            float xv = x[col[e]];
            acc = fmaf(val[e], xv, acc);
            double p = (double)val[e] * (double)xv;   /* exact in binary64 */
            a64 += p;
            s64 += fabs(p);
        }
        y32[r] = acc;
        y64[r] = a64;
        asum[r] = s64;
    }
}

/* ------------------------------------------------------------ pointer chase */

void or_pchase(const int32_t* next, const int32_t* start, int32_t* end, int64_t nchasers,
               int64_t hops) {
    for (int64_t t = 0; t < nchasers; ++t) {
        int32_t p = start[t];
        for (int64_t h = 0; h < hops; ++h) p = next[p];
        end[t] = p;
    }
}

/* ------------------------------------------------------------ triad: a = s*c + b, fused */

void or_triad(const float* b, const float* c, float* a, float s, int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) a[i] = fmaf(s, c[i], b[i]);
}

/* ------------------------------------------------------------ 256-bin histogram */

void or_hist256(const uint8_t* data, uint32_t* hist, int64_t n) {
    for (int v = 0; v < 256; ++v) hist[v] = 0;
    for (int64_t i = 0; i < n; ++i) hist[data[i]] += 1;
}

/* ------------------------------------------------------------ escape-time
 * pixel (i,j): cx = x0 + (j+0.5)*dx, cy = y0 + (i+0.5)*dy; z0 = 0;
 * iterate while it < max_iter: stop when x^2 + y^2 > 4, else
 * y <- 2xy + cy, x <- x^2 - y^2 + cx (every operation rounded separately). */

void or_escape(uint32_t* count, int64_t width, int64_t height, int64_t max_iter, float x0,
               float y0, float dx, float dy, int64_t row_lo, int64_t row_hi) {
    for (int64_t i = row_lo; i < row_hi; ++i)
        for (int64_t j = 0; j < width; ++j) {
            float tj = (float)j + 0.5f;
            float ti = (float)i + 0.5f;
            float ox = tj * dx;
            float oy = ti * dy;
            float cx = x0 + ox;
            float cy = y0 + oy;
            float x = 0.0f, y = 0.0f;
            int64_t it = 0;
            while (it < max_iter) {
                float x2 = x * x;
                float y2 = y * y;
                float r2 = x2 + y2;
                if (r2 > 4.0f) break;
                float xy = x * y;
                float xy2 = xy + xy;
                y = xy2 + cy;
                float d = x2 - y2;
                x = d + cx;
                ++it;
            }
            count[i * width + j] = (uint32_t)it;
        }
}

/* ------------------------------------------------------------ sort (the definition:
 * the ascending permutation of the input) */

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

void or_sort_u32(const uint32_t* in, uint32_t* out, int64_t n) {
    memcpy(out, in, (size_t)n * 4);
    qsort(out, (size_t)n, 4, cmp_u32);
}

/* ------------------------------------------------------------ MatrixAdd (Section 4.1 example) */

void or_matadd(const float* a, const float* b, float* c, int64_t n) {
    for (int64_t i = 0; i < n * n; ++i) c[i] = a[i] + b[i];
}


/* ------------------------------------------------------------ TEA */
/* Tiny Encryption Algorithm (D. Wheeler, R. Needham, "TEA, a Tiny Encryption
 * Algorithm", FSE 1994): 32 cycles; each cycle adds the key-schedule
 * constant 0x9E3779B9 to sum, then updates v0 from v1 and v1 from v0, all
 * modulo 2^32. Block j is (words[2j], words[2j+1]). */
void or_tea(const uint32_t* words, uint32_t* out, const uint32_t* key, int64_t n) {
  for (int64_t j = 0; j < n; ++j) {
    uint32_t v0 = words[2 * j], v1 = words[2 * j + 1], sum = 0;
    for (int c = 0; c < 32; ++c) {
      sum += 0x9E3779B9u;
      v0 += ((v1 << 4) + key[0]) ^ (v1 + sum) ^ ((v1 >> 5) + key[1]);
      v1 += ((v0 << 4) + key[2]) ^ (v0 + sum) ^ ((v0 >> 5) + key[3]);
    }
    out[2 * j] = v0;
    out[2 * j + 1] = v1;
  }
}

/* ------------------------------------------------------------ SAD */
/* For every 4x4 block (bx, by) of the current frame, in row-major block
 * order, and every displacement (dx, dy) in [-R, R]^2 (dy major): the sum over
 * the block's 16 pixels of |cur - ref| with the reference pixel at the
 * displaced position, coordinates clamped into the frame. */
void or_sad(const uint8_t* cur, const uint8_t* ref, uint32_t* sad, int64_t W, int64_t H, int64_t R) {
  const int64_t D = 2 * R + 1;
  int64_t o = 0;
  for (int64_t by = 0; by < H / 4; ++by)
    for (int64_t bx = 0; bx < W / 4; ++bx)
      for (int64_t dy = -R; dy <= R; ++dy)
        for (int64_t dx = -R; dx <= R; ++dx) {
          uint32_t acc = 0;
          for (int64_t i = 0; i < 4; ++i)
            for (int64_t j = 0; j < 4; ++j) {
              int64_t y = 4 * by + i, x = 4 * bx + j;
              int64_t ry = y + dy < 0 ? 0 : (y + dy > H - 1 ? H - 1 : y + dy);
              int64_t rx = x + dx < 0 ? 0 : (x + dx > W - 1 ? W - 1 : x + dx);
              int d = (int)cur[y * W + x] - (int)ref[ry * W + rx];
              acc += (uint32_t)(d < 0 ? -d : d);
            }
          sad[o++] = acc;
        }
  (void)D;
}

/* ------------------------------------------------------------ 3-D stencil */
/* 7-point stencil on an nz x ny x nx grid (x fastest): interior points
 * c0 * c + c1 * s with s = ((((w + e) + n) + s) + b) + t over the six face
 * neighbours (-x, +x, -y, +y, -z, +z), each addition rounded, then
 * fmaf(c1, s, c0 * c); points on the grid's faces are copied. */
void or_stencil7(const float* in, float* out, int64_t nx, int64_t ny, int64_t nz, float c0, float c1) {
  const int64_t sy = nx, sz = nx * ny;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        const int64_t i = z * sz + y * sy + x;
        if (x == 0 || y == 0 || z == 0 || x == nx - 1 || y == ny - 1 || z == nz - 1) {
          out[i] = in[i];
          continue;
        }
        float s = in[i - 1] + in[i + 1];
        s = s + in[i - sy];
        s = s + in[i + sy];
        s = s + in[i - sz];
        s = s + in[i + sz];
        out[i] = fmaf(c1, s, c0 * in[i]);
      }
}

/* ------------------------------------------------------------ MRI-Q */
/* sine and cosine of a binary32 angle: Cody-Waite reduction a = n pi/2 + r
 * with pi/2 in two parts (1.57079637f, -4.37113900e-8f) and n the nearest
 * integer to a * 2/pi; Taylor polynomials of sin (to r^9) and cos (to r^8)
 * on |r| <= pi/4 in Horner form with fmaf; the quadrant n mod 4 swaps and
 * negates them. */
void or_sincosf(float a, float* sn, float* cs) {
  const float n = rintf(a * 0.636619772f);
  float r = fmaf(-n, 1.57079637f, a);
  r = fmaf(-n, -4.37113900e-8f, r);
  const float r2 = r * r;
  float ps = fmaf(r2, 2.75573192e-6f, -1.98412698e-4f);
  ps = fmaf(r2, ps, 8.33333333e-3f);
  ps = fmaf(r2, ps, -1.66666667e-1f);
  const float s = fmaf(r * r2, ps, r);
  float pc = fmaf(r2, 2.48015873e-5f, -1.38888889e-3f);
  pc = fmaf(r2, pc, 4.16666667e-2f);
  pc = fmaf(r2, pc, -0.5f);
  const float c = fmaf(r2, pc, 1.0f);
  switch (((int)n) & 3) {
    case 0: *sn = s; *cs = c; break;
    case 1: *sn = c; *cs = -s; break;
    case 2: *sn = -s; *cs = -c; break;
    default: *sn = -c; *cs = s; break;
  }
}

/* phiMag[k] = fmaf(phiI, phiI, phiR * phiR); for each point x:
 * Qr = sum_k phiMag[k] cos(2 pi (k . x)), Qi likewise with sin, k ascending,
 * each term fmaf(phiMag, cos, Qr); k . x = fmaf(kz, z, fmaf(ky, y, kx * x));
 * the angle is 6.28318548f (binary32 2 pi) times it, rounded.
 * Points [lo, hi) only, so tests can sample large cases. */
void or_mriq(const float* kx, const float* ky, const float* kz, const float* phiR, const float* phiI,
             float* phiMag, const float* x, const float* y, const float* z, float* Qr, float* Qi, int64_t numK,
             const int64_t* pts, int64_t npts) {
  for (int64_t k = 0; k < numK; ++k) phiMag[k] = fmaf(phiI[k], phiI[k], phiR[k] * phiR[k]);
  for (int64_t p = 0; p < npts; ++p) {
    const int64_t i = pts[p];
    float qr = 0.0f, qi = 0.0f;
    for (int64_t k = 0; k < numK; ++k) {
      float t = kx[k] * x[i];
      t = fmaf(ky[k], y[i], t);
      t = fmaf(kz[k], z[i], t);
      float sn, cs;
      or_sincosf(6.28318548f * t, &sn, &cs);
      qr = fmaf(phiMag[k], cs, qr);
      qi = fmaf(phiMag[k], sn, qi);
    }
    Qr[p] = qr;
    Qi[p] = qi;
  }
}
