// Two-qubit gates of any kind as one-qubit gates around a canonical gate
// (host code behind cc_kak_gates).
//
// Every two-qubit unitary U (Schmidt rank 4 in general, Eq. 1) factors as
//   U = e^{i g} (A1 (x) B1) CAN(tx, ty, tz) (A0 (x) B0)
// with one-qubit unitaries A, B and CAN(tx, ty, tz) = exp(-i (tx XX + ty YY +
// tz ZZ) / 2): the Cartan (KAK) decomposition (Khaneja and Glaser 2001, Kraus
// and Cirac 2001).  In the magic (Bell) basis M, local unitaries become real
// orthogonal matrices and CAN becomes diagonal, so with Ub = M^dag U M (U
// scaled to determinant 1) the symmetric unitary Ub^T Ub = P D P^T is
// diagonalised by a real orthogonal P (found from a generic real combination
// of its real and imaginary parts, a real symmetric matrix, by cyclic Jacobi
// rotations), and Ub = K1 D^{1/2} P^T with K1 real orthogonal.
//
// Convention: a 4x4 matrix on (q0, q1) acts on |x_q0 x_q1>, index 2 x_q0 + x_q1.
#include <cmath>
#include <complex>
#include <cstring>

#include "internal.h"

namespace cc {
namespace {

using M4 = cd[4][4];
using M2 = cd[2][2];
const double kPi = 3.14159265358979323846;

void mul4(const M4 a, const M4 b, M4 out) {
  M4 t;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  std::memcpy(out, t, sizeof(M4));
}

void adjoint4(const M4 a, M4 out) {
  M4 t;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) t[i][j] = std::conj(a[j][i]);
  std::memcpy(out, t, sizeof(M4));
}

void transpose4(const M4 a, M4 out) {
  M4 t;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) t[i][j] = a[j][i];
  std::memcpy(out, t, sizeof(M4));
}

// Determinant by Gaussian elimination with partial pivoting.
cd det4(const M4 a) {
  M4 m;
  std::memcpy(m, a, sizeof(M4));
  cd det = 1.0;
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::abs(m[r][c]) > std::abs(m[p][c])) p = r;
    if (std::abs(m[p][c]) == 0.0) return 0.0;
    if (p != c) {
      for (int k = 0; k < 4; ++k) std::swap(m[p][k], m[c][k]);
      det = -det;
    }
    det *= m[c][c];
    for (int r = c + 1; r < 4; ++r) {
      const cd f = m[r][c] / m[c][c];
      for (int k = c; k < 4; ++k) m[r][k] -= f * m[c][k];
    }
  }
  return det;
}

// The magic basis (columns).
void magic(M4 m) {
  const double h = 1.0 / std::sqrt(2.0);
  const cd I(0.0, 1.0);
  const cd v[4][4] = {{1.0, 0.0, 0.0, I}, {0.0, I, 1.0, 0.0}, {0.0, I, -1.0, 0.0},
                      {1.0, 0.0, 0.0, -I}};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m[i][j] = v[i][j] * h;
}

// Eigenvectors (columns of p) of a real symmetric 4x4 matrix by cyclic Jacobi
// rotations (Golub and Van Loan, Sec. 8.5).
void jacobi_eigenvectors(double a[4][4], double p[4][4]) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) p[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        tot += a[i][j] * a[i][j];
        if (i != j) off += a[i][j] * a[i][j];
      }
    if (off <= 1e-32 * tot || off == 0.0) return;
    for (int r = 0; r < 3; ++r)
      for (int s = r + 1; s < 4; ++s) {
        if (a[r][s] == 0.0) continue;
        const double theta = (a[s][s] - a[r][r]) / (2.0 * a[r][s]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::abs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < 4; ++k) {  // A <- A J
          const double akr = a[k][r], aks = a[k][s];
          a[k][r] = c * akr - sn * aks;
          a[k][s] = sn * akr + c * aks;
        }
        for (int k = 0; k < 4; ++k) {  // A <- J^T A
          const double ark = a[r][k], ask = a[s][k];
          a[r][k] = c * ark - sn * ask;
          a[s][k] = sn * ark + c * ask;
        }
        for (int k = 0; k < 4; ++k) {  // P <- P J
          const double pkr = p[k][r], pks = p[k][s];
          p[k][r] = c * pkr - sn * pks;
          p[k][s] = sn * pkr + c * pks;
        }
      }
  }
}

void can_matrix(double tx, double ty, double tz, M4 out) {
  // exp(-i (tx XX + ty YY + tz ZZ) / 2) on |x_q0 x_q1>: XX swaps 00 <-> 11 and
  // 01 <-> 10; YY does the same with signs -1 (00, 11) and +1 (01, 10); ZZ is
  // diag(1, -1, -1, 1).  The three commute; the closed form per block:
  const cd I(0.0, 1.0);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) out[i][j] = 0.0;
  // block {00, 11}: XX - YY = 2 X_block on it, ZZ = +1
  const double a = (tx - ty) / 2.0, b = (tx + ty) / 2.0;
  const cd ez = std::exp(-I * tz / 2.0), ezi = std::exp(I * tz / 2.0);
  out[0][0] = ez * std::cos(a);
  out[0][3] = -I * ez * std::sin(a);
  out[3][0] = -I * ez * std::sin(a);
  out[3][3] = ez * std::cos(a);
  // block {01, 10}: XX + YY = 2 X_block on it, ZZ = -1
  out[1][1] = ezi * std::cos(b);
  out[1][2] = -I * ezi * std::sin(b);
  out[2][1] = -I * ezi * std::sin(b);
  out[2][2] = ezi * std::cos(b);
}

// A, B with A (x) B = k for a 4x4 matrix known to be a tensor product: the
// realigned matrix r[(a0 a1)][(b0 b1)] = k[2 a0 + b0][2 a1 + b1] is rank 1,
// vec(A) vec(B)^T; both factors are scaled to |det| = 1.
void split_local(const M4 k, M2 A, M2 B) {
  cd r[4][4];
  for (int a0 = 0; a0 < 2; ++a0)
    for (int a1 = 0; a1 < 2; ++a1)
      for (int b0 = 0; b0 < 2; ++b0)
        for (int b1 = 0; b1 < 2; ++b1) r[2 * a0 + a1][2 * b0 + b1] = k[2 * a0 + b0][2 * a1 + b1];
  int pi = 0, pj = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (std::abs(r[i][j]) > std::abs(r[pi][pj])) {
        pi = i;
        pj = j;
      }
  for (int i = 0; i < 4; ++i) A[i >> 1][i & 1] = r[i][pj];
  for (int j = 0; j < 4; ++j) B[j >> 1][j & 1] = r[pi][j] / r[pi][pj];
  const double da = std::sqrt(std::abs(A[0][0] * A[1][1] - A[0][1] * A[1][0]));
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      A[i][j] /= da;
      B[i][j] *= da;
    }
}

void kron2(const M2 a, const M2 b, M4 out) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) out[i][j] = a[i >> 1][j >> 1] * b[i & 1][j & 1];
}

void u3m(double th, double ph, double la, M2 out) {
  const cd I(0.0, 1.0);
  const double c = std::cos(th / 2), s = std::sin(th / 2);
  out[0][0] = c;
  out[0][1] = -std::exp(I * la) * s;
  out[1][0] = std::exp(I * ph) * s;
  out[1][1] = std::exp(I * (ph + la)) * c;
}

// (theta, phi, lambda, g) with u = e^{i g} U3(theta, phi, lambda): theta from
// the entry magnitudes, phi + lambda from u11 conj(u00), phi - lambda from
// u10 conj(-u01); halving leaves (phi, lambda) ambiguous by (pi, pi), which
// flips both off-diagonal signs, so the candidate that reproduces u is kept.
void u3_params(const M2 u, double& th, double& ph, double& la, double& g) {
  const double c_abs = 0.5 * (std::abs(u[0][0]) + std::abs(u[1][1]));
  const double s_abs = 0.5 * (std::abs(u[0][1]) + std::abs(u[1][0]));
  th = 2.0 * std::atan2(s_abs, c_abs);
  const double sigma = c_abs > 0 ? std::arg(u[1][1] * std::conj(u[0][0])) : 0.0;
  const double delta = s_abs > 0 ? std::arg(u[1][0] * std::conj(-u[0][1])) : 0.0;
  double best = 1e300;
  for (int k = 0; k < 2; ++k) {
    const double p = 0.5 * (sigma + delta) + k * kPi, l = 0.5 * (sigma - delta) + k * kPi;
    M2 b;
    u3m(th, p, l, b);
    const int i = 0, j = c_abs >= s_abs ? 0 : 1;
    const double gg = std::arg(u[i][j] / b[i][j]);
    const cd e = std::exp(cd(0.0, gg));
    double err = 0.0;
    for (int r = 0; r < 2; ++r)
      for (int q = 0; q < 2; ++q) err = std::max(err, std::abs(e * b[r][q] - u[r][q]));
    if (err < best) {
      best = err;
      ph = p;
      la = l;
      g = gg;
    }
  }
}

cc_gate make_gate(int kind, int q0, int q1, double th, double ph, double la) {
  cc_gate x{};
  x.kind = kind;
  x.q0 = q0;
  x.q1 = q1;
  x.theta = th;
  x.phi = ph;
  x.lambda = la;
  return x;
}

}  // namespace
}  // namespace cc

extern "C" cc_status cc_kak_gates(const double* u_interleaved, int32_t q0, int32_t q1,
                                  cc_gate* out, int32_t* n_out) {
  using namespace cc;
  if (!u_interleaved || !out || !n_out) return fail(CC_EINVAL, "cc_kak_gates: NULL argument");
  if (q0 < 0 || q1 < 0 || q0 == q1 || q0 >= CC_MAX_QUBITS || q1 >= CC_MAX_QUBITS)
    return fail(CC_EINVAL, "cc_kak_gates: need two distinct qubits in range");
  M4 u;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) u[i][j] = cd(u_interleaved[8 * i + 2 * j], u_interleaved[8 * i + 2 * j + 1]);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (!std::isfinite(u[i][j].real()) || !std::isfinite(u[i][j].imag()))
        return fail(CC_EINVAL, "cc_kak_gates: matrix entries must be finite");
  {  // unitarity
    M4 ud, p;
    adjoint4(u, ud);
    mul4(ud, u, p);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (std::abs(p[i][j] - cd(i == j ? 1.0 : 0.0)) > 1e-10)
          return fail(CC_EINVAL, "cc_kak_gates: the matrix is not unitary");
  }
  const cd I(0.0, 1.0);
  const double g0 = std::arg(det4(u)) / 4.0;
  M4 up, M, Md, ub, ubt, m2;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) up[i][j] = u[i][j] * std::exp(-I * g0);
  magic(M);
  adjoint4(M, Md);
  mul4(Md, up, ub);
  mul4(ub, M, ub);
  transpose4(ub, ubt);
  mul4(ubt, ub, m2);  // symmetric unitary
  // a generic real combination of Re m2 and Im m2 has the common eigenvectors
  static const double kComb[8][2] = {{0.8, 0.6},   {-0.3, 1.1}, {1.3, -0.7}, {0.45, 0.9},
                                     {-1.2, -0.5}, {0.2, -1.4}, {1.7, 0.35}, {-0.6, 0.75}};
  double P[4][4];
  cd d[4];
  bool found = false;
  for (const auto& ab : kComb) {
    double s[4][4];
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) s[i][j] = ab[0] * m2[i][j].real() + ab[1] * m2[i][j].imag();
    jacobi_eigenvectors(s, P);
    // check that P^T m2 P is diagonal
    double off = 0.0;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        cd x = 0.0;
        for (int k = 0; k < 4; ++k)
          for (int l = 0; l < 4; ++l) x += P[k][i] * m2[k][l] * P[l][j];
        if (i == j) d[i] = x;
        else off = std::max(off, std::abs(x));
      }
    if (off < 1e-9) {
      found = true;
      break;
    }
  }
  if (!found) return fail(CC_EUNSUPPORTED, "cc_kak_gates: simultaneous diagonalisation failed");
  {  // det P = +1
    M4 pc;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) pc[i][j] = P[i][j];
    if (det4(pc).real() < 0)
      for (int i = 0; i < 4; ++i) P[i][0] = -P[i][0];
  }
  double half[4];
  for (int j = 0; j < 4; ++j) half[j] = std::arg(d[j]) / 2.0;
  M4 Pc, k1;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) Pc[i][j] = P[i][j];
  auto make_k1 = [&]() {
    M4 dh;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) dh[i][j] = i == j ? std::exp(-I * half[i]) : cd(0.0);
    mul4(ub, Pc, k1);
    mul4(k1, dh, k1);
  };
  make_k1();
  if (det4(k1).real() < 0) {  // move a pi into one eigenphase
    half[0] += kPi;
    make_k1();
  }
  M4 k2, a1b1, a0b0;
  transpose4(Pc, k2);
  mul4(M, k1, a1b1);
  mul4(a1b1, Md, a1b1);
  mul4(M, k2, a0b0);
  mul4(a0b0, Md, a0b0);
  // half_j = g1 - (tx sx_j + ty sy_j + tz sz_j) / 2 with s_pj = <M_j|P (x) P|M_j>;
  // in the magic basis these signs are fixed, so the 4 x 4 system is solved
  // by elimination
  double sys[4][5];
  for (int j = 0; j < 4; ++j) {
    sys[j][0] = 1.0;
    for (int p = 0; p < 3; ++p) {
      // XX|x> = |x ^ 3>, YY|x> = -(-1)^{popc x}|x ^ 3>, ZZ|x> = (-1)^{popc x}|x>
      cd e = 0.0;
      for (int x = 0; x < 4; ++x) {
        const double par = ((x >> 1) ^ x) & 1 ? -1.0 : 1.0;
        cd v;
        if (p == 0) v = M[x ^ 3][j];
        else if (p == 1) v = -par * M[x ^ 3][j];
        else v = par * M[x][j];
        e += std::conj(M[x][j]) * v;
      }
      sys[j][1 + p] = -0.5 * e.real();
    }
    sys[j][4] = half[j];
  }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::abs(sys[r][c]) > std::abs(sys[p][c])) p = r;
    for (int k = 0; k < 5; ++k) std::swap(sys[p][k], sys[c][k]);
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = sys[r][c] / sys[c][c];
      for (int k = c; k < 5; ++k) sys[r][k] -= f * sys[c][k];
    }
  }
  const double g1 = sys[0][4] / sys[0][0];
  const double tx = sys[1][4] / sys[1][1], ty = sys[2][4] / sys[2][2], tz = sys[3][4] / sys[3][3];
  {  // the middle factor must be e^{i g1} CAN(tx, ty, tz)
    M4 mid, dh, can;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) dh[i][j] = i == j ? std::exp(I * half[i]) : cd(0.0);
    mul4(M, dh, mid);
    mul4(mid, Md, mid);
    can_matrix(tx, ty, tz, can);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (std::abs(mid[i][j] - std::exp(I * g1) * can[i][j]) > 1e-9)
          return fail(CC_EUNSUPPORTED, "cc_kak_gates: canonical parameters do not reproduce the middle factor");
  }
  M2 A0, B0, A1, B1;
  split_local(a1b1, A1, B1);
  split_local(a0b0, A0, B0);
  // the remaining global phase (each split is exact up to a scalar)
  M4 l0, l1, can, lhs;
  kron2(A0, B0, l0);
  kron2(A1, B1, l1);
  can_matrix(tx, ty, tz, can);
  mul4(can, l0, lhs);
  mul4(l1, lhs, lhs);
  int bi = 0, bj = 0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (std::abs(lhs[i][j]) > std::abs(lhs[bi][bj])) {
        bi = i;
        bj = j;
      }
  double phase = std::arg(u[bi][bj] / lhs[bi][bj]);
  int n = 0;
  const M2* locals[4] = {&A0, &B0, &A1, &B1};
  const int qs[4] = {q0, q1, q0, q1};
  for (int k = 0; k < 4; ++k) {
    double th, ph, la, gg;
    u3_params(*locals[k], th, ph, la, gg);
    phase += gg;
    out[n++] = make_gate(CC_GATE_U3, qs[k], -1, th, ph, la);
    if (k == 1) out[n++] = make_gate(CC_GATE_CAN, q0, q1, tx, ty, tz);
  }
  phase = std::remainder(phase, 2 * kPi);
  if (std::abs(phase) > 1e-15) {  // P X P X = e^{i g} I for P = diag(1, e^{i g})
    out[n++] = make_gate(CC_GATE_U3, q0, -1, 0.0, 0.0, phase);
    out[n++] = make_gate(CC_GATE_X, q0, -1, 0.0, 0.0, 0.0);
    out[n++] = make_gate(CC_GATE_U3, q0, -1, 0.0, 0.0, phase);
    out[n++] = make_gate(CC_GATE_X, q0, -1, 0.0, 0.0, 0.0);
  }
  *n_out = n;
  return CC_OK;
}
