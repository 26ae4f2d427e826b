// Core-set certificates for the certified SVM search (see coreset.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/pdscp.h"

namespace pdscp {

constexpr int kCoresetK = 512;       // points per class picked by one direction
constexpr int kCoresetRounds = 4;    // active-set rounds of one check
constexpr int kCoresetMaxPerClass = 4 * kCoresetK;  // core-set size cap per class
constexpr int64_t kCoresetFirst = 256;  // first check at this many iterations of the search, then every doubling

// Exact polytope distance of two small point sets (host, FP64) by a primal
// active-set method; returns the iterations run. mu (nP), ga (nQ): the
// weights on the two simplices; z (d): P^T mu - Q^T ga; *gap: z.z minus
// (min_i p_i.z - max_j q_j.z) at the end (>= 0; <= tol z.z when converged).
// mu0, ga0 (optional): weights to start from (their positive entries are the
// first support, renormalised per class), e.g. a previous solution on a
// subset of the points.
int pd_active_set(const double* P, int nP, const double* Q, int nQ, int d, double tol, int max_iter, double* mu,
                  double* ga, double* z, double* gap, const double* mu0 = nullptr, const double* ga0 = nullptr);

// Bytes of workspace the core-set checks of svm_solve need for n points in d.
size_t coreset_bytes(int64_t n, int d);

// One core-set check (core-set certificates, a reading beyond the paper):
// from direction w0 (host, d doubles), core sets picked on the device,
// solved on the host.
// Sets *lb (a margin of some direction over all points), *ub (a core-set
// distance) and w_lb (that direction, unit norm). ws: coreset_bytes(n, d)
// bytes of device memory, 256-byte aligned.
// The SES counterpart (points, no radii): the core set is the K farthest
// points from centre c0 (host, d doubles), then from each new centre; *lb =
// sqrt(phi) of the Frank-Wolfe dual weights on the core set (weak duality of
// the enclosing-ball QP), *ub the radius over every point of the ball at the
// best centre found, c_ub that centre. Same workspace as the SVM check.
pdscp_status ses_coreset_check(const void* X, int dtype, int64_t n, int d, const double* c0, double eps, void* ws,
                               cudaStream_t s, double* lb, double* ub, std::vector<double>& c_ub);

pdscp_status svm_coreset_check(const void* X, int dtype, const int8_t* y, int64_t n, int d, const double* w0,
                               double eps, void* ws, cudaStream_t s, double* lb, double* ub,
                               std::vector<double>& w_lb);

}  // namespace pdscp
