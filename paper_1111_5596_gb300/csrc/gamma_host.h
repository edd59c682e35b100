// Host-side DeGrand-Rossi gamma matrices as exact complex integers, shared by
// the contraction launchers (mesons, baryons).  The basis is the QDP++ chiral
// basis: gamma_1..gamma_4 Hermitian, Gamma(n) = g1^n0 g2^n1 g3^n2 g4^n3,
// Gamma(15) = gamma_5 = diag(1, 1, -1, -1), charge conjugation C = g2 g4.
#pragma once

namespace qdpg {
namespace gamma_host {

struct CInt {
  int re, im;
};
inline CInt operator*(CInt a, CInt b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline CInt operator+(CInt a, CInt b) { return {a.re + b.re, a.im + b.im}; }
inline CInt conj(CInt a) { return {a.re, -a.im}; }

struct Mat4 {
  CInt m[4][4];
};

inline Mat4 mat_mul(const Mat4& a, const Mat4& b) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      CInt s{0, 0};
      for (int k = 0; k < 4; ++k) s = s + a.m[i][k] * b.m[k][j];
      c.m[i][j] = s;
    }
  return c;
}

// gamma_1..gamma_4 of the DeGrand-Rossi (QDP++ chiral) basis, listed by the
// single nonzero of each row: column and value.
inline Mat4 basis_gamma(int mu) {
  static const int col[4][4] = {{3, 2, 1, 0}, {3, 2, 1, 0}, {2, 3, 0, 1}, {2, 3, 0, 1}};
  static const CInt val[4][4] = {
      {{0, 1}, {0, 1}, {0, -1}, {0, -1}},   // gamma_1
      {{-1, 0}, {1, 0}, {1, 0}, {-1, 0}},   // gamma_2
      {{0, 1}, {0, -1}, {0, -1}, {0, 1}},   // gamma_3
      {{1, 0}, {1, 0}, {1, 0}, {1, 0}}};    // gamma_4
  Mat4 g{};
  for (int r = 0; r < 4; ++r) g.m[r][col[mu][r]] = val[mu][r];
  return g;
}

inline Mat4 Gamma(int n) {
  Mat4 g{};
  for (int i = 0; i < 4; ++i) g.m[i][i] = {1, 0};
  for (int bit = 0; bit < 4; ++bit)
    if ((n >> bit) & 1) g = mat_mul(g, basis_gamma(bit));
  return g;
}

inline Mat4 dagger(const Mat4& a) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) c.m[i][j] = conj(a.m[j][i]);
  return c;
}

// XOR mask of a signed permutation (row r -> column r ^ mask); -1 if none.
inline int xor_mask(const Mat4& a) {
  int mask = -1;
  for (int c = 0; c < 4; ++c)
    if (a.m[0][c].re || a.m[0][c].im) mask = c;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      bool nz = a.m[r][c].re || a.m[r][c].im;
      if (nz != (c == (r ^ mask))) return -1;
    }
  return mask;
}


inline Mat4 charge_conj() { return mat_mul(basis_gamma(1), basis_gamma(3)); }

}  // namespace gamma_host
}  // namespace qdpg
