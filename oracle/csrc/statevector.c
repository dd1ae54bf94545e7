/*
 * O1 state-vector kernels for the FP64 oracle (test infrastructure only).
 *
 * psi is a complex128 vector of length 2^n stored as interleaved (re, im)
 * doubles; qubit 0 is the most significant bit of the index, so qubit q sits
 * at bit position n-1-q.  A gate U[out][in] acts on the amplitudes that differ
 * only in its qubits' bits: psi'[.., o, ..] = sum_i U[o][i] psi[.., i, ..]
 * (the definition of applying a gate to one or two qubits of a register; paper
 * Fig. 1 circuit model).  Plain loops, no blocking; OpenMP splits the
 * independent groups of amplitudes.
 */
#include <stdint.h>

typedef struct { double re, im; } cplx;

static inline cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static inline cplx cadd(cplx a, cplx b) {
  cplx r = {a.re + b.re, a.im + b.im};
  return r;
}

/* u: 2x2 row-major complex [out][in] as 8 doubles. */
void sv_apply_1q(double *psi_d, int n, int q, const double *u_d) {
  cplx *psi = (cplx *)psi_d;
  const cplx *u = (const cplx *)u_d;
  const int64_t bit = (int64_t)1 << (n - 1 - q);
  const int64_t half = (int64_t)1 << (n - 1);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < half; ++k) {
    /* k enumerates indices with the target bit removed; insert a 0 there */
    int64_t i0 = ((k & ~(bit - 1)) << 1) | (k & (bit - 1));
    int64_t i1 = i0 | bit;
    cplx a0 = psi[i0], a1 = psi[i1];
    psi[i0] = cadd(cmul(u[0], a0), cmul(u[1], a1));
    psi[i1] = cadd(cmul(u[2], a0), cmul(u[3], a1));
  }
}

/* u: 4x4 row-major complex [out][in] on |q_a q_b>, q_a most significant. */
void sv_apply_2q(double *psi_d, int n, int qa, int qb, const double *u_d) {
  cplx *psi = (cplx *)psi_d;
  const cplx *u = (const cplx *)u_d;
  const int64_t ba = (int64_t)1 << (n - 1 - qa);
  const int64_t bb = (int64_t)1 << (n - 1 - qb);
  const int64_t lo = ba < bb ? ba : bb, hi = ba < bb ? bb : ba;
  const int64_t quarter = (int64_t)1 << (n - 2);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < quarter; ++k) {
    int64_t t = ((k & ~(lo - 1)) << 1) | (k & (lo - 1));
    int64_t i00 = ((t & ~(hi - 1)) << 1) | (t & (hi - 1));
    int64_t idx[4] = {i00, i00 | bb, i00 | ba, i00 | ba | bb}; /* basis |a b> = 0,1,2,3 */
    cplx in[4];
    for (int j = 0; j < 4; ++j) in[j] = psi[idx[j]];
    for (int o = 0; o < 4; ++o) {
      cplx acc = {0.0, 0.0};
      for (int j = 0; j < 4; ++j) acc = cadd(acc, cmul(u[4 * o + j], in[j]));
      psi[idx[o]] = acc;
    }
  }
}

/* psi <- |0...0> */
void sv_zero_state(double *psi_d, int n) {
  const int64_t len = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < 2 * len; ++i) psi_d[i] = 0.0;
  psi_d[0] = 1.0;
}
