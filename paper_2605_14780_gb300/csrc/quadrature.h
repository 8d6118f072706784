// Reconstruction-and-quadrature rows of cubed-sphere edge ghosts (the
// finite-volume form of the user-defined interpolation of Sec. II-B, written
// as Itp = Agg . Recons in Sec. III-B), lowered to user CSR sub-matrices on
// the host at plan creation.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/bc.h"
#include "prune.h"

namespace bcg {

// True if one of the sub-matrices asks for BC_GEOM_CUBED_SPHERE_QUAD rows.
bool has_cs_quadrature(const bc_submatrix* subs, int nsubs);

// Copies the list into `out`, every BC_INTERP sub-matrix of geometry
// BC_GEOM_CUBED_SPHERE_QUAD replaced by the BC_CSR sub-matrices of its rows
// (one for the scalar components, one for the vector pair), in place of it.
// Other sub-matrices are copied unchanged.  On failure returns the status and
// sets `msg`.
bc_status lower_cs_quadrature(const bc_grid* grid, const bc_submatrix* subs, int nsubs,
                              SubStore& out, std::string& msg);

// Gauss-Legendre nodes (ascending) and weights of n points on [-1, 1].
void gauss_legendre(int n, double* x, double* w);

// Weights c[0..p) of the polynomial of degree p - 1 whose averages over the
// unit cells [k - 1/2, k + 1/2] are given, evaluated at x.
void average_reconstruction(double x, int p, double* c);

}  // namespace bcg
