// Host-side integer lattice layer: Smith normal form of M and the exact index
// maps between the stored FFT grid and the pattern P(M) / generating set
// G(M^T) of the paper's Sec. 2.1.
//
// The pattern DFT of Eq. (Fouriermatrix) pairs y in P(M) with h in G(M^T)
// through exp(-2 pi i h^T y).  With U M V = S = diag(s_1..s_d) (U, V
// unimodular), y = M^-1 U^-1 n and h = V^-T l give
// h^T y = l^T V^-1 M^-1 U^-1 n = l^T S^-1 n, so the DFT becomes an ordinary
// d-dimensional DFT over the grid Z_{s_1} x .. x Z_{s_d}.  Reductions into the
// half-open cube [-1/2,1/2)^d are done exactly on integer numerators over
// m = |det M|.

#include <algorithm>
#include <cstdlib>
#include <string>
#include <utility>

#include "internal.hpp"

namespace fh {

namespace {

bool mul_ok(int64_t a, int64_t b, int64_t* out) { return !__builtin_mul_overflow(a, b, out); }
bool add_ok(int64_t a, int64_t b, int64_t* out) { return !__builtin_add_overflow(a, b, out); }

// floor(a / b) for b > 0
int64_t floordiv(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// extended gcd: g = x a + y b, g >= 0
int64_t ext_gcd(int64_t a, int64_t b, int64_t* x, int64_t* y) {
  int64_t x0 = 1, y0 = 0, x1 = 0, y1 = 1;
  while (b != 0) {
    int64_t q = a / b;
    int64_t t = a - q * b; a = b; b = t;
    t = x0 - q * x1; x0 = x1; x1 = t;
    t = y0 - q * y1; y0 = y1; y1 = t;
  }
  if (a < 0) { a = -a; x0 = -x0; y0 = -y0; }
  *x = x0; *y = y0;
  return a;
}

int64_t det3(const int64_t A[3][3], int d) {
  if (d == 2) return A[0][0] * A[1][1] - A[0][1] * A[1][0];
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

void adjugate(const int64_t A[3][3], int d, int64_t out[3][3]) {
  if (d == 2) {
    out[0][0] = A[1][1]; out[0][1] = -A[0][1];
    out[1][0] = -A[1][0]; out[1][1] = A[0][0];
    return;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // cofactor C_ji goes to out[i][j]
      int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (i + 1) % 3, c1 = (i + 2) % 3;
      out[i][j] = A[r0][c0] * A[r1][c1] - A[r0][c1] * A[r1][c0];
    }
}

// Unimodular 2x2 transform of rows (p, q): [row_p; row_q] <- [[x, y], [-b/g, a/g]] [row_p; row_q]
template <int N>
void row_bezout(int64_t A[3][3], int64_t T[3][3], int d, int p, int q, int64_t x, int64_t y,
                int64_t bg, int64_t ag) {
  for (int c = 0; c < d; ++c) {
    int64_t ap = A[p][c], aq = A[q][c];
    A[p][c] = x * ap + y * aq;
    A[q][c] = -bg * ap + ag * aq;
    int64_t tp = T[p][c], tq = T[q][c];
    T[p][c] = x * tp + y * tq;
    T[q][c] = -bg * tp + ag * tq;
  }
}

template <int N>
void col_bezout(int64_t A[3][3], int64_t T[3][3], int d, int p, int q, int64_t x, int64_t y,
                int64_t bg, int64_t ag) {
  for (int r = 0; r < d; ++r) {
    int64_t ap = A[r][p], aq = A[r][q];
    A[r][p] = x * ap + y * aq;
    A[r][q] = -bg * ap + ag * aq;
    int64_t tp = T[r][p], tq = T[r][q];
    T[r][p] = x * tp + y * tq;
    T[r][q] = -bg * tp + ag * tq;
  }
}

// Bezout coefficients for eliminating b against the pivot a: g = x a + y b.
// With divisor_first, a pivot that divides b gives the plain elimination
// step (x, y, g) = (1, 0, a), which leaves the pivot's row or column as it is.
// The extended-gcd step alone can return (0, +-1) when |a| = |b|, a swap that
// the following column (row) step undoes, so the elimination can cycle.
int64_t bezout(int64_t a, int64_t b, bool divisor_first, int64_t* x, int64_t* y) {
  if (divisor_first && b % a == 0) { *x = 1; *y = 0; return a; }
  return ext_gcd(a, b, x, y);
}

// Smith normal form by Bezout eliminations: U A V = diag.  Returns false for a
// singular matrix or when the elimination did not finish within its guard.
// With divisor_first every step either clears its entry without touching
// the pivot's row (column) or replaces the pivot by a gcd of strictly smaller
// magnitude, and a divisibility fix-up is followed by such a step, so the
// elimination ends.
bool smith(const int64_t M[3][3], int d, bool divisor_first, int64_t U[3][3], int64_t V[3][3],
           int64_t S[3]) {
  int64_t A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      A[i][j] = (i < d && j < d) ? M[i][j] : 0;
      U[i][j] = V[i][j] = (i == j);
    }
  for (int t = 0; t < d; ++t) {
    bool done = false;
    for (int guard = 0; guard < 10000 && !done; ++guard) {
      // bring a nonzero entry of the trailing block to (t,t)
      if (A[t][t] == 0) {
        int bi = -1, bj = -1;
        for (int i = t; i < d && bi < 0; ++i)
          for (int j = t; j < d; ++j)
            if (A[i][j] != 0) { bi = i; bj = j; break; }
        if (bi < 0) return false;
        for (int c = 0; c < d; ++c) { std::swap(A[t][c], A[bi][c]); std::swap(U[t][c], U[bi][c]); }
        for (int r = 0; r < d; ++r) { std::swap(A[r][t], A[r][bj]); std::swap(V[r][t], V[r][bj]); }
      }
      // clear column t below the pivot
      for (int i = t + 1; i < d; ++i) {
        if (A[i][t] == 0) continue;
        int64_t x, y, a = A[t][t], b = A[i][t];
        int64_t g = bezout(a, b, divisor_first, &x, &y);
        row_bezout<0>(A, U, d, t, i, x, y, b / g, a / g);
      }
      // clear row t right of the pivot
      for (int j = t + 1; j < d; ++j) {
        if (A[t][j] == 0) continue;
        int64_t x, y, a = A[t][t], b = A[t][j];
        int64_t g = bezout(a, b, divisor_first, &x, &y);
        col_bezout<0>(A, V, d, t, j, x, y, b / g, a / g);
      }
      bool clean = true;
      for (int i = t + 1; i < d; ++i) clean = clean && A[i][t] == 0;
      if (!clean) continue;
      // divisibility: the pivot must divide the trailing block
      int bad = -1;
      for (int i = t + 1; i < d && bad < 0; ++i)
        for (int j = t + 1; j < d; ++j)
          if (A[i][j] % A[t][t] != 0) { bad = i; break; }
      if (bad < 0) { done = true; break; }
      for (int c = 0; c < d; ++c) { A[t][c] += A[bad][c]; U[t][c] += U[bad][c]; }
    }
    if (!done) return false;
    if (A[t][t] < 0)
      for (int c = 0; c < d; ++c) { A[t][c] = -A[t][c]; U[t][c] = -U[t][c]; }
  }
  for (int i = 0; i < d; ++i) S[i] = A[i][i];
  return true;
}

void reduce_numerators(int64_t* a, int d, int64_t D) {
  for (int i = 0; i < d; ++i) a[i] -= D * floordiv(2 * a[i] + D, 2 * D);
}

}  // namespace

int64_t Pattern::half_len() const { return dims[nd - 1] / 2 + 1; }

int64_t Pattern::n_half() const {
  int64_t n = half_len();
  for (int k = 0; k < nd - 1; ++k) n *= dims[k];
  return n;
}

void Pattern::point_numerator(int64_t idx, int64_t* a) const {
  int64_t j[3] = {0, 0, 0};
  for (int k = nd - 1; k >= 0; --k) {
    int64_t n = idx % dims[k];
    idx /= dims[k];
    for (int i = 0; i < d; ++i) j[i] += n * Pmap[k][i];
  }
  for (int i = 0; i < d; ++i) {
    int64_t s = 0;
    for (int c = 0; c < d; ++c) s += adj[i][c] * j[c];
    a[i] = sign * s;
  }
  reduce_numerators(a, d, D);
}

void Pattern::half_freq(int64_t idx, int64_t* h) const {
  int64_t hl = half_len();
  int64_t l[3] = {0, 0, 0};
  l[nd - 1] = idx % hl;
  idx /= hl;
  for (int k = nd - 2; k >= 0; --k) { l[k] = idx % dims[k]; idx /= dims[k]; }
  for (int i = 0; i < d; ++i) {
    h[i] = 0;
    for (int k = 0; k < nd; ++k) h[i] += l[k] * Fmap[k][i];
  }
  int64_t u[3];
  for (int i = 0; i < d; ++i) {
    int64_t s = 0;
    for (int c = 0; c < d; ++c) s += adjT[i][c] * h[c];
    u[i] = sign * s;
  }
  int64_t z[3];
  for (int i = 0; i < d; ++i) z[i] = floordiv(2 * u[i] + D, 2 * D);
  for (int i = 0; i < d; ++i)
    for (int c = 0; c < d; ++c) h[i] -= M[c][i] * z[c];  // h - M^T z
}

fh_status build_pattern(int d, const int64_t* Min, Pattern* out) {
  if (d != 2 && d != 3) { set_error("d must be 2 or 3"); return FH_ERR_ARG; }
  Pattern P;
  P.d = d;
  int64_t maxabs = 0;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      P.M[i][j] = Min[i * d + j];
      maxabs = std::max<int64_t>(maxabs, std::llabs(P.M[i][j]));
    }
  // |entries| <= 2^20 keeps every product below in int64 for d <= 3.
  if (maxabs > (int64_t(1) << 20)) { set_error("|M_ij| > 2^20"); return FH_ERR_OVERFLOW; }
  int64_t det = det3(P.M, d);
  if (det == 0) { set_error("M is singular"); return FH_ERR_SINGULAR_M; }
  P.sign = det > 0 ? 1 : -1;
  P.D = det > 0 ? det : -det;
  if (P.D >= (int64_t(1) << 31)) { set_error("|det M| >= 2^31"); return FH_ERR_OVERFLOW; }
  adjugate(P.M, d, P.adj);
  int64_t Mt[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Mt[i][j] = P.M[j][i];
  adjugate(Mt, d, P.adjT);
  // The extended-gcd elimination first (it fixes the storage layout of every
  // pattern it handles); the divisor-first variant for the matrices on which
  // it cycles, e.g. [[6, 4], [14, 10]].
  if (!smith(P.M, d, false, P.U, P.V, P.snf) && !smith(P.M, d, true, P.U, P.V, P.snf)) {
    set_error("Smith normal form failed");
    return FH_ERR_INTERNAL;
  }
  int64_t du = det3(P.U, d), dv = det3(P.V, d);
  if ((du != 1 && du != -1) || (dv != 1 && dv != -1)) { set_error("SNF transforms not unimodular"); return FH_ERR_INTERNAL; }
  adjugate(P.U, d, P.Uinv);
  adjugate(P.V, d, P.Vinv);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) { P.Uinv[i][j] *= du; P.Vinv[i][j] *= dv; }
  // check U M V = S
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      int64_t s = 0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) s += P.U[i][a] * P.M[a][b] * P.V[b][j];
      if (s != (i == j ? P.snf[i] : 0)) { set_error("SNF check failed"); return FH_ERR_INTERNAL; }
    }
  // storage axes: non-trivial SNF factors in increasing order (SNF already
  // orders them by divisibility), the last one contiguous
  P.nd = 0;
  for (int i = 0; i < d; ++i)
    if (P.snf[i] > 1) { P.axis_of[P.nd] = i; P.dims[P.nd] = int(P.snf[i]); ++P.nd; }
  if (P.nd == 0) { P.nd = 1; P.axis_of[0] = d - 1; P.dims[0] = 1; }
  for (int k = 0; k < P.nd; ++k)
    for (int i = 0; i < d; ++i) {
      P.Pmap[k][i] = P.Uinv[i][P.axis_of[k]];   // column of U^-1
      P.Fmap[k][i] = P.Vinv[P.axis_of[k]][i];   // row of V^-1 = column of V^-T
    }
  // overflow bound for the device-side maps: |h| <= sum_k |Fmap| dims
  int64_t hb = 0;
  for (int i = 0; i < d; ++i) {
    int64_t s = 0;
    for (int k = 0; k < P.nd; ++k) {
      int64_t t;
      if (!mul_ok(std::llabs(P.Fmap[k][i]), P.dims[k], &t) || !add_ok(s, t, &s)) {
        set_error("frequency map overflows"); return FH_ERR_OVERFLOW;
      }
    }
    hb = std::max(hb, s);
  }
  int64_t ab = 0;
  for (int i = 0; i < d; ++i)
    for (int c = 0; c < d; ++c) ab = std::max<int64_t>(ab, std::llabs(P.adjT[i][c]));
  int64_t t1, t2;
  if (!mul_ok(hb + maxabs * 4, ab, &t1) || !mul_ok(t1, 3 * 4, &t2) || t2 > (int64_t(1) << 60)) {
    set_error("index maps could overflow int64"); return FH_ERR_OVERFLOW;
  }
  *out = P;
  return FH_OK;
}

// Radix plan: largest supported radices first (8, 4, 2 for the power of two,
// then 3, 5, 7, 11, 13).
bool make_plan(int L, FftPlan* plan) {
  FftPlan p;
  p.L = L;
  int n = L;
  auto push = [&](int r) { if (p.np >= 24) return false; p.r[p.np++] = r; n /= r; return true; };
  while (n % 8 == 0) if (!push(8)) return false;
  while (n % 4 == 0) if (!push(4)) return false;
  while (n % 2 == 0) if (!push(2)) return false;
  for (int r : {3, 5, 7, 11, 13})
    while (n % r == 0) if (!push(r)) return false;
  // larger primes: the generic direct-DFT stage
  for (int r = 17; r * r <= n; r += 2)
    while (n % r == 0) if (!push(r)) return false;
  if (n > 1 && !push(n)) return false;
  *plan = p;
  return true;
}

}  // namespace fh
