/*
 * Oracle (test infrastructure only): exact product of two non-negative integers
 * held as little-endian arrays of uint64 limbs, and the low / high products
 * obtained from it by their definitions (Section 1 of the paper: the low product
 * is uv mod 2^n; a high product is any 0 <= w <= 2^n with |uv - 2^n w| < 2^n).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this
 * file. It shares nothing with the CUDA library.
 *
 * Method: schoolbook below KARA_CUTOFF limbs, Karatsuba above, with the three
 * half-size products of the top `par_depth` levels run on POSIX threads.
 * 64x64 -> 128-bit limb products use unsigned __int128.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;
#define KARA_CUTOFF 32

/* r[0 .. na+nb) = a[0 .. na) * b[0 .. nb) */
static void mul_school(uint64_t* r, const uint64_t* a, size_t na,
                       const uint64_t* b, size_t nb) {
  memset(r, 0, (na + nb) * sizeof(uint64_t));
  for (size_t i = 0; i < na; ++i) {
    uint64_t ai = a[i], carry = 0;
    for (size_t j = 0; j < nb; ++j) {
      u128 t = (u128)ai * b[j] + r[i + j] + carry;
      r[i + j] = (uint64_t)t;
      carry = (uint64_t)(t >> 64);
    }
    r[i + nb] = carry;
  }
}

/* r[0..n] = a[0..n) + b[0..m), m <= n; returns nothing, r has n+1 limbs */
static void add_ext(uint64_t* r, const uint64_t* a, size_t n, const uint64_t* b, size_t m) {
  uint64_t c = 0;
  for (size_t i = 0; i < n; ++i) {
    u128 t = (u128)a[i] + (i < m ? b[i] : 0) + c;
    r[i] = (uint64_t)t;
    c = (uint64_t)(t >> 64);
  }
  r[n] = c;
}

/* x[0..n) -= y[0..m), m <= n; the true difference is non-negative */
static void sub_in(uint64_t* x, size_t n, const uint64_t* y, size_t m) {
  uint64_t borrow = 0;
  for (size_t i = 0; i < n; ++i) {
    uint64_t yi = i < m ? y[i] : 0;
    uint64_t d = x[i] - yi - borrow;
    borrow = (x[i] < yi) || (x[i] - yi < borrow);
    x[i] = d;
    if (i >= m && !borrow) break;
  }
}

/* x[0..n) += y[0..m), m <= n; carry out of x is dropped (caller sizes x) */
static void add_in(uint64_t* x, size_t n, const uint64_t* y, size_t m) {
  uint64_t c = 0;
  for (size_t i = 0; i < n; ++i) {
    if (i >= m && !c) break;
    u128 t = (u128)x[i] + (i < m ? y[i] : 0) + c;
    x[i] = (uint64_t)t;
    c = (uint64_t)(t >> 64);
  }
}

static void kara(uint64_t* r, const uint64_t* a, const uint64_t* b, size_t n, int par_depth);

typedef struct { uint64_t* r; const uint64_t* a; const uint64_t* b; size_t n; int depth; } kjob;
static void* kara_thread(void* p) {
  kjob* j = (kjob*)p;
  kara(j->r, j->a, j->b, j->n, j->depth);
  return NULL;
}

/* r[0 .. 2n) = a[0..n) * b[0..n) */
static void kara(uint64_t* r, const uint64_t* a, const uint64_t* b, size_t n, int par_depth) {
  if (n < KARA_CUTOFF) { mul_school(r, a, n, b, n); return; }
  size_t h = n / 2, m = n - h;           /* a = a0 + B^h a1, |a0| = h, |a1| = m >= h */
  uint64_t* sa = (uint64_t*)malloc((m + 1) * sizeof(uint64_t));
  uint64_t* sb = (uint64_t*)malloc((m + 1) * sizeof(uint64_t));
  uint64_t* z1 = (uint64_t*)malloc(2 * (m + 1) * sizeof(uint64_t));
  add_ext(sa, a + h, m, a, h);           /* sa = a0 + a1 */
  add_ext(sb, b + h, m, b, h);
  /* z0 = a0 b0 into r[0 .. 2h), z2 = a1 b1 into r[2h .. 2n), z1 = sa sb */
  if (par_depth > 0) {
    pthread_t t0, t2;
    kjob j0 = {r, a, b, h, par_depth - 1}, j2 = {r + 2 * h, a + h, b + h, m, par_depth - 1};
    int ok0 = pthread_create(&t0, NULL, kara_thread, &j0) == 0;
    if (!ok0) kara_thread(&j0);
    int ok2 = pthread_create(&t2, NULL, kara_thread, &j2) == 0;
    if (!ok2) kara_thread(&j2);
    kara(z1, sa, sb, m + 1, par_depth - 1);
    if (ok0) pthread_join(t0, NULL);
    if (ok2) pthread_join(t2, NULL);
  } else {
    kara(r, a, b, h, 0);
    kara(r + 2 * h, a + h, b + h, m, 0);
    kara(z1, sa, sb, m + 1, 0);
  }
  /* z1 -= z0 + z2 ; the middle term a0 b1 + a1 b0 fits in 2m+1 limbs */
  sub_in(z1, 2 * (m + 1), r, 2 * h);
  sub_in(z1, 2 * (m + 1), r + 2 * h, 2 * m);
  /* r += z1 * B^h */
  add_in(r + h, 2 * n - h, z1, 2 * m + 1 < 2 * n - h ? 2 * m + 1 : 2 * n - h);
  free(sa); free(sb); free(z1);
}

/* Full product: out[0 .. 2*nl) = u[0..nl) * v[0..nl). */
void oracle_mul_full(uint64_t* out, const uint64_t* u, const uint64_t* v, size_t nl, int par_depth) {
  if (nl == 0) return;
  kara(out, u, v, nl, par_depth);
}

static size_t ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

/* Low product (definition): out[0 .. ceil(n/64)) = (u v) mod 2^n. */
void oracle_mul_lo(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits, int par_depth) {
  size_t nl = ceil_div(n_bits, 64);
  uint64_t* full = (uint64_t*)malloc(2 * nl * sizeof(uint64_t));
  oracle_mul_full(full, u, v, nl, par_depth);
  memcpy(out, full, nl * sizeof(uint64_t));
  if (n_bits % 64) out[nl - 1] &= (((uint64_t)1) << (n_bits % 64)) - 1;
  free(full);
}

/* High product accept-set (definition): out[0 .. floor(n/64)+1) = q = floor(u v / 2^n);
 * *rem_nonzero = 1 iff u v mod 2^n != 0, in which case q + 1 is also a valid
 * high product (|uv - 2^n (q+1)| < 2^n); otherwise only q is. */
void oracle_mul_hi_floor(uint64_t* out, int* rem_nonzero, const uint64_t* u, const uint64_t* v,
                         uint64_t n_bits, int par_depth) {
  size_t nl = ceil_div(n_bits, 64), no = n_bits / 64 + 1;
  uint64_t* full = (uint64_t*)calloc(2 * nl + 1, sizeof(uint64_t));
  oracle_mul_full(full, u, v, nl, par_depth);
  size_t w = n_bits / 64; unsigned s = (unsigned)(n_bits % 64);
  for (size_t j = 0; j < no; ++j) {
    uint64_t lo = (w + j < 2 * nl) ? full[w + j] : 0;
    uint64_t hi = (w + j + 1 < 2 * nl) ? full[w + j + 1] : 0;
    out[j] = s ? ((lo >> s) | (hi << (64 - s))) : lo;
  }
  int nz = 0;
  for (size_t i = 0; i < w && !nz; ++i) nz = full[i] != 0;
  if (!nz && s) nz = (full[w] & ((((uint64_t)1) << s) - 1)) != 0;
  *rem_nonzero = nz;
  free(full);
}
