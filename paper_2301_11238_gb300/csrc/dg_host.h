// Host-side setup for the DG shallow-water / regularized-Bingham library:
// reference-element operators of the nodal basis and mesh connectivity.
//
// Everything here runs once per context (not timed).  Element operators are
// those of a nodal Lagrange basis on equispaced nodes, evaluated with the
// quadrature rules the library fixes for the weak form of Sec. 5
// (Eq. WeakForm51/52): Gauss-Legendre on lines, collapsed Gauss-Legendre x
// Gauss-Jacobi(1,0) on triangles, ceil(3p/2) points per direction in volumes
// and ceil((3p+1)/2) on edges.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#if defined(__CUDACC__)
#define DG_HOST_DEVICE __host__ __device__
#else
#define DG_HOST_DEVICE
#endif

namespace dgswe {

// rows of the per-element geometry array: dr_a/dx_i (4), J, dx (step-bound
// length), 1/J (precomputed so the kernels divide by J nowhere)
constexpr int kGeoRows = 7;


// Element-local index of node k of face f in the equispaced nodal ordering.
// 1D: nodes 0..p from left to right; face 0 is the left end, face 1 the
// right.  Triangles: node (i, j), i + j <= p, has index
// sum_{jj < j} (p + 1 - jj) + i; face 0 is j = 0, face 1 is i + j = p and
// face 2 is i = 0, each walked counter-clockwise.  The kernels evaluate it
// with compile-time arguments, so the node indices become constants.
DG_HOST_DEVICE constexpr int face_node(int dim, int p, int f, int k) {
  if (dim == 1) return f == 0 ? 0 : p;
  int i = 0, j = 0;
  if (f == 0) {
    i = k;
    j = 0;
  } else if (f == 1) {
    i = p - k;
    j = k;
  } else {
    i = 0;
    j = p - k;
  }
  int base = 0;
  for (int jj = 0; jj < j; ++jj) base += p + 1 - jj;
  return base + i;
}

// Gauss-Jacobi rule for weight (1-x)^a (1+x)^b on [-1,1] by Golub-Welsch.
void gauss_jacobi(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);

struct RefOps {
  int dim = 0, p = 0;
  int Np = 0, Nq = 0, nf = 0, Nfp = 0, Nfq = 0;
  std::vector<double> rnodes;   // Np x dim, equispaced node coordinates
  std::vector<double> rq, wq;   // Nq x dim, Nq
  std::vector<double> Vq;       // Nq x Np   l_a at volume points
  std::vector<double> Drq, Dsq; // Nq x Np   dl_a/dr, dl_a/ds at volume points
  std::vector<double> Dr, Ds;   // Np x Np   nodal differentiation
  std::vector<double> M, Minv;  // Np x Np   reference mass matrix and inverse
  std::vector<double> wint;     // Np        integral of l_a over the reference element
  std::vector<int> fmask;       // nf x Nfp  element node index of face node k
  std::vector<double> tf, wf;   // Nfq       edge quadrature parameters / weights
  std::vector<double> Lf;       // Nfq x Nfp edge Lagrange (face nodes) at edge points
  std::vector<double> LIFT;     // Np x (nf*Nfp)  M^-1 * (face mass on face nodes)
};

bool build_refops(int dim, int p, RefOps& ops, std::string& err);

// Source coefficients of the bed and slope terms of Eq. Sterm at the volume
// quadrature points: c_j = -g_c dH/dx_j - g_s delta_1j, so that the source of
// momentum equation j is S_j = h c_j.  The bed H is the element's nodal
// interpolant; geo is the [kGeoRows][K] geometry.  Layout [dim * Nq][K].
void build_bed_source(int dim, const RefOps& ops, int64_t K, const std::vector<double>& geo,
                      const std::vector<double>& bed, double gc, double gs, std::vector<double>& src);

// Geometry and connectivity of a conforming mesh of intervals (dim 1) or
// counter-clockwise triangles (dim 2).
struct MeshData {
  int dim = 0, nf = 0;
  int64_t K = 0, F = 0;                     // elements, unique faces
  std::vector<double> geo;                  // [kGeoRows][K]: G00 G01 G10 G11 (dr_a/dx_i), J, dx, 1/J
  std::vector<int32_t> nbr;                 // [nf][K] neighbour element, or -1-bc for boundary
  std::vector<int8_t> nbrf;                 // [nf][K] neighbour's local face
  std::vector<int32_t> fid;                 // [nf][K] face id; bit 31 set when not the owner
  std::vector<double> fn;                   // [nf][dim][K] outward unit normal
  std::vector<double> fsj;                  // [nf][K] face Jacobian (length / 2; 1 in 1D)
  std::vector<int32_t> face_e1, face_e2;    // [F] owner element; other element or -1-bc
  std::vector<int8_t> face_f1, face_f2;     // [F] local faces
  std::vector<double> face_n;               // [dim][F] owner's outward normal
  std::vector<double> face_sj;              // [F]
  std::vector<double> node_xyz;             // [K][Np][dim] physical node coordinates
};

bool build_mesh(int dim, int64_t n_vertices, const double* coords, int64_t n_elements,
                const int32_t* etov, const int8_t* face_bc, int n_bc, const RefOps& ops,
                MeshData& m, std::string& err);

}  // namespace dgswe
