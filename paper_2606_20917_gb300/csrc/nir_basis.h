// nir_basis.h -- host-side FP64 quadrature, basis and interpolation tables.
#pragma once

double nirb_jacobi(int n, double a, double b, double x);
double nirb_jacobi_d(int n, double a, double b, double x);
// Gauss-Jacobi rule (Golub-Welsch) for the weight (1-x)^a (1+x)^b, ascending.
bool nirb_gauss_jacobi(int Q, double a, double b, double *z, double *w);
// Gauss-Lobatto-Legendre rule with Q points (Q >= 2), ascending.
bool nirb_gll(int Q, double *z, double *w);
double nirb_psiA(int p, double z);
double nirb_psiB(int p, int q, double z);
// Collocation derivative matrix D[i*Q + j] = l_j'(z_i).
void nirb_colloc(int Q, const double *z, double *D);
// Equispaced-lattice Lagrange values and derivatives at z: L[q*(g+1) + a].
void nirb_lagrange_equi(int g, int Q, const double *z, double *L, double *dL);
// Per-direction points and weights of a shape (collapse factors in w).
bool nirb_shape_rules(int shape, int Q, double *z /*[3][Q]*/, double *w /*[3][Q]*/);
// Fill the kernel table blob (layout in nir_layout.h) in FP64; basis 0: the
// modified expansion, 1: GLL-Lagrange in reflection-pair form (quad/hex).
bool nirb_build_tables(int shape, int P, int Q, double *blob, int basis);
double nirb_nodal_pair(int p, int N, double z);
int nirb_table_size(int shape, int P, int Q);
