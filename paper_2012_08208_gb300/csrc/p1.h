// Private: the paper's P1 cells on the structured grid (cell shapes, their
// unit-modulus matrices and the midpoint-filter stencil), shared by the P1
// operator entry point and the P1 problem handle.
#pragma once

namespace tp {

constexpr int kP1MaxTypes = 6;  // 4 triangle shapes (2D), 6 Kuhn tetrahedra (3D)
constexpr int kP1MaxNd = 12;    // DOFs of a tetrahedron

// Unit-modulus cell matrices (row-major, dim (dim + 1) rows; DOF order vertex
// then component) and vertex offsets within the square / cube of every cell
// shape.  They travel with each launch as part of a kernel's __grid_constant__
// parameter block (about 7.2 KB, within the 32 KB parameter limit), so
// concurrent calls with different materials cannot see each other's matrices.
struct P1Shapes {
  double K[kP1MaxTypes][kP1MaxNd * kP1MaxNd];
  int off[kP1MaxTypes][4][3];
};

// Vertex offsets of shape `type`.  2D: 0, 1 = the cells of a square cut along
// (0,0)-(1,1); 2, 3 = cut along (1,0)-(0,1).  3D: the Kuhn path of the t-th
// axis ordering in lexicographic order.
void p1_shape_offsets(int dim, int type, int off[4][3]);
// Fill K and off for every shape; returns the shape count (4 or 6).
int p1_shapes(int dim, double lam, double mu, double K[kP1MaxTypes][kP1MaxNd * kP1MaxNd],
              int off[kP1MaxTypes][4][3]);
// Midpoint-filter stencil per centre shape: entries (dx, dy, dz, local cell)
// and weights rmin - distance (> 0), grouped by shape, count[t] per shape.
// Returns the entry count, or -1 when it exceeds cap.
int p1_filter_stencil(int dim, int diagonal, double rmin, int cap, int* count, int (*ent)[4], double* w);

}  // namespace tp
