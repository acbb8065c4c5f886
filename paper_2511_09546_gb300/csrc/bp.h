// Mean-field (chi = 1) metric preconditioner (Sec. III.B, App. A); see bp.cu.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "common.h"
#include "ipeps_impl.h"

namespace ipeps {

// Sweep limits the optimiser uses for the mean-field metric
constexpr double kBpTol = 1e-12;
constexpr int kBpMaxit = 1000;

// The converged messages of a cell, their eigendecompositions and the
// per-site norms <A|1 (x) m_u (x) m_l (x) m_d (x) m_r|A>, all on the device.
struct BpMetric {
  Cell cell;
  int sweeps = 0;
  double change = INFINITY;
  DBuf msgs;  // 4 * nsites messages, D x D each, index (x * Ly + y) * 4 + leg (u, l, d, r)
  DBuf V;     // eigenvectors of each message, row-major, column j = eigenvector j
  DBuf lam;   // eigenvalues, D per message
  DBuf nrm;   // one per site
};

// Message sweeps from identity / D until no entry changes by more than tol
// (or maxit sweeps), then the eigendecompositions and norms.  Throws
// IPEPS_ERR_NONFINITE if a message loses its positive trace.
void bp_metric(const Cell &c, const double *A, double tol, int maxit, BpMetric &m, cudaStream_t s);
// out = (N + delta I)^-1 g for every tensor of the cell (g, out: device, layout of A)
void bp_apply(const BpMetric &m, const double *g, double delta, double *out, cudaStream_t s);

}  // namespace ipeps
