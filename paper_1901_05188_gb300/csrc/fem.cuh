// Device-side finite-element arithmetic (Sec. 2): orthotropic Hooke law,
// ply rotation and blocks of the trilinear hexahedral element stiffness.
#pragma once

#include "common.cuh"

namespace geneo {

// Voigt index of the symmetric pair (i, j): order 11, 22, 33, 23, 13, 12.
__device__ __forceinline__ int voigt(int i, int j) {
  // table {{0,5,4},{5,1,3},{4,3,2}} packed 3 bits per entry
  const unsigned t = 0u | (5u << 3) | (4u << 6) | (5u << 9) | (1u << 12) | (3u << 15) |
                     (4u << 18) | (3u << 21) | (2u << 24);
  return (t >> (3 * (3 * i + j))) & 7u;
}

// 6x6 stiffness (row-major) of an orthotropic material in its own axes:
// invert the compliance built from the nine engineering constants (Sec. 2).
__device__ inline void material_stiffness(const geneo_ortho &m, double C[36]) {
  double S[36];
  for (int i = 0; i < 36; ++i) S[i] = 0.0;
  S[0] = 1.0 / m.E1;
  S[7] = 1.0 / m.E2;
  S[14] = 1.0 / m.E3;
  S[1] = S[6] = -m.nu12 / m.E1;
  S[2] = S[12] = -m.nu13 / m.E1;
  S[8] = S[13] = -m.nu23 / m.E2;
  S[21] = 1.0 / m.G23;
  S[28] = 1.0 / m.G13;
  S[35] = 1.0 / m.G12;
  // Gauss-Jordan with partial pivoting on [S | I]
  double Aug[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) Aug[i][j] = j < 6 ? S[6 * i + j] : (j - 6 == i ? 1.0 : 0.0);
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    for (int r = c + 1; r < 6; ++r)
      if (fabs(Aug[r][c]) > fabs(Aug[piv][c])) piv = r;
    if (piv != c)
      for (int j = 0; j < 12; ++j) {
        double t = Aug[c][j];
        Aug[c][j] = Aug[piv][j];
        Aug[piv][j] = t;
      }
    double inv = 1.0 / Aug[c][c];
    for (int j = 0; j < 12; ++j) Aug[c][j] *= inv;
    for (int r = 0; r < 6; ++r) {
      if (r == c) continue;
      double f = Aug[r][c];
      for (int j = 0; j < 12; ++j) Aug[r][j] -= f * Aug[c][j];
    }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) C[6 * i + j] = Aug[i][6 + j];
}

// Rotate a Voigt stiffness from ply axes to global axes with the stress
// transformation (Bond) matrix M of Q = R_z(theta) R_y(phi): C' = M C M^T.
// The fibre direction Q e1 is (cos t cos p, sin t cos p, -sin p).
__device__ inline void rotate_voigt(const double C[36], double theta, double phi, double Cr[36]) {
  double ct = cos(theta), st = sin(theta), cp = cos(phi), sp = sin(phi);
  // Q = Rz * Ry
  double Q[3][3] = {{ct * cp, -st, ct * sp}, {st * cp, ct, st * sp}, {-sp, 0.0, cp}};
  const int VI[6] = {0, 1, 2, 1, 0, 0};
  const int VJ[6] = {0, 1, 2, 2, 2, 1};
  double M[36];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      int i = VI[I], j = VJ[I], k = VI[J], l = VJ[J];
      double v = Q[i][k] * Q[j][l];
      if (k != l) v += Q[i][l] * Q[j][k];
      M[6 * I + J] = v;
    }
  double T[36];
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double s = 0.0;
      for (int K = 0; K < 6; ++K) s += M[6 * I + K] * C[6 * K + J];
      T[6 * I + J] = s;
    }
  for (int I = 0; I < 6; ++I)
    for (int J = 0; J < 6; ++J) {
      double s = 0.0;
      for (int K = 0; K < 6; ++K) s += T[6 * I + K] * M[6 * J + K];
      Cr[6 * I + J] = s;
    }
}

// Integral over the box element of d_j N_a * d_l N_b (trilinear N, axis-aligned
// box of sides h): a product over the axes of 1D integrals of the linear
// factors, with s = +-1 the slope sign of a factor and 1/h its derivative's
// size: int f_a f_b = h/3 (same side) or h/6, int f_a' f_b = s_a/2,
// int f_a f_b' = s_b/2, int f_a' f_b' = s_a s_b / h.  The 2x2x2 Gauss rule is
// exact for these products, so this equals the quadrature to rounding.
__device__ __forceinline__ double box_grad_integral(const double sa[3], const double sb[3],
                                                    const double h[3], const double ih[3],
                                                    int j, int l) {
  double v = 1.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double f;
    if (d == j && d == l) f = sa[d] * sb[d] * ih[d];
    else if (d == j) f = 0.5 * sa[d];
    else if (d == l) f = 0.5 * sb[d];
    else f = (sa[d] == sb[d] ? (1.0 / 3.0) : (1.0 / 6.0)) * h[d];
    v *= f;
  }
  return v;
}

// 3x3 block K_ab of the Q1 element stiffness of an hx x hy x hz box with
// global-frame Voigt stiffness C (row-major 6x6):
//   K_ab[i][k] = sum_{j,l} C_ijkl G_ab[j][l],  G_ab[j][l] = int dN_a/dx_j dN_b/dx_l,
// the integrals in closed form, equal to the 2x2x2 Gauss-Legendre rule (Sec. 2).
// Local node a sits at corner (a & 1, (a >> 1) & 1, (a >> 2) & 1).
__device__ inline void element_block(const double *__restrict__ C, double hx, double hy,
                                     double hz, int a, int b, double K[9]) {
  const double sa[3] = {double(2 * (a & 1) - 1), double(2 * ((a >> 1) & 1) - 1),
                        double(2 * ((a >> 2) & 1) - 1)};
  const double sb[3] = {double(2 * (b & 1) - 1), double(2 * ((b >> 1) & 1) - 1),
                        double(2 * ((b >> 2) & 1) - 1)};
  const double h[3] = {hx, hy, hz};
  const double ih[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
  double G[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int l = 0; l < 3; ++l) G[j][l] = box_grad_integral(sa, sb, h, ih, j, l);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) s += C[6 * voigt(i, j) + voigt(k, l)] * G[j][l];
      K[3 * i + k] = s;
    }
}

// int K grad N_a . grad N_b over an hx x hy x hz box with K = diag(kd), in closed
// form, equal to 2x2x2 Gauss points (local node a at corner (a & 1, (a >> 1) & 1, a >> 2)).
__device__ inline double darcy_entry(const double *__restrict__ kd, double hx, double hy,
                                     double hz, int a, int b) {
  const double sa[3] = {double(2 * (a & 1) - 1), double(2 * ((a >> 1) & 1) - 1),
                        double(2 * ((a >> 2) & 1) - 1)};
  const double sb[3] = {double(2 * (b & 1) - 1), double(2 * ((b >> 1) & 1) - 1),
                        double(2 * ((b >> 2) & 1) - 1)};
  const double h[3] = {hx, hy, hz};
  const double ih[3] = {1.0 / hx, 1.0 / hy, 1.0 / hz};
  return kd[0] * box_grad_integral(sa, sb, h, ih, 0, 0) +
         kd[1] * box_grad_integral(sa, sb, h, ih, 1, 1) +
         kd[2] * box_grad_integral(sa, sb, h, ih, 2, 2);
}

}  // namespace geneo
