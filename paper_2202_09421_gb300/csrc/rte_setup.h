// Host-side FP64 set-up of the FC-DOM operators and boundary tables.
// Internal to the library; the kernels receive FP32 copies.
#pragma once
#include <vector>

namespace rte_setup {

constexpr double kPi = 3.14159265358979323846;
constexpr double kTieTol = 1e-12;

// Smallest N >= n whose prime factors are all <= 5 (Sec. 4.3: E extra zeros).
int smooth5(int n);

// Dense FC derivative operator D (n x n, row-major D[i*n + j]) of a line of n
// points at spacing h: continuation with the FC-Gram table (d = 5, C = 25),
// filtered spectral derivative of eqs. (RTEFCSum)-(RTEFCSumder) with period
// N_p h, Nyquist mode dropped.  Built as D = (circulant kernel) * (extension).
void fc_derivative_matrix(int n, double h, double alpha, double beta,
                          std::vector<double>& D);

// The decomposed operator of Sec. 4.4 / Algorithm 1: the n points split
// into `parts` owned ranges [k n / parts, (k + 1) n / parts), each extended
// by two fringe points on interior sides; row i of D is the row of i's owner
// in the FC operator of the owner's segment (columns of that segment).
// parts <= 1 is fc_derivative_matrix.  Returns false if a segment has fewer
// than 16 points.
bool fc_derivative_matrix_parts(int n, double h, double alpha, double beta, int parts,
                                std::vector<double>& D);
// Owned range [lo, hi) and segment [slo, shi) of part k of `parts` (two
// fringe points on each interior side).
void part_range(int n, int parts, int k, int& lo, int& hi, int& slo, int& shi);
// Largest spectral-radius estimate over the segments of a decomposition.
double fc_spectral_radius_parts(int n, double h, double alpha, double beta, int parts);

// Split, pre-swizzled image of D for the tcgen05 kernels: for every chunk q
// of 32 input positions, a hi tile then a lo tile, each n_rows (= n rounded
// up to 128) rows x 32 tf32 values in the K-major 128-byte-swizzle order
// (value (i, kk) at i*32 + ((kk/4) ^ (i%8))*4 + kk%4); hi = tf32(D),
// lo = tf32(D - hi), zero padding outside n x n.
void tc_operator_image(const std::vector<double>& D, int n, std::vector<float>& img);

// BF16 form of the same image: chunks of 64 input positions, each a hi then
// a lo tile of n_rows x 64 bf16 values (value (i, kk) at
// i*64 + ((kk/8) ^ (i%8))*8 + kk%8); hi = bf16(D), lo = bf16(D - hi), both
// rounded to nearest even.
void tc_operator_image_bf16(const std::vector<double>& D, int n, std::vector<unsigned short>& img);

// Same split and swizzle for the phase matrix as the scattering operand:
// rows m, K = q, 32 x 32 (zero-padded) hi tile then lo tile.
void tc_phase_image(const std::vector<double>& P, int M, std::vector<float>& img);

// Segment operator of one part of the decomposed operator (Sec. 4.4) as the
// B operand of the tensor-core fused step: rows i < hi - lo (owned points),
// K = box position p = s + (slo - lo + 2) for segment point s < shi - slo
// (the box starts two points before the owned range), 16 rows x 32 tf32 in
// the K-major 128-byte-swizzle order, a hi tile then a lo tile (1024 floats
// written to img); entries outside the segment are zero.
void tc_segment_image(const std::vector<double>& D, int n, int lo, int hi, int slo, int shi, float* img);

// Largest |multiplier| of the filtered periodic derivative on N_p points,
// the spectral-radius estimate of D used by the stability check.
double fc_spectral_radius(int n, double h, double alpha, double beta);

// Normalised phase matrix Pt[m*M + m'] = w p_{m,m'} (Sec. 4.1).
void phase_matrix(int M, double g, double exponent, std::vector<double>& P);

// Unpolarised Fresnel reflectance at incidence cosine |cos_i|, n_in -> n_out.
double fresnel(double cos_i, double n_in, double n_out);

// Window function of eq. (sourcelabwind).
double window(double v);

// Boundary tables.  Faces: 0 left (x = xmin), 1 right, 2 bottom (y = ymin),
// 3 top.  Corners: 0 (left, bottom), 1 (right, bottom), 2 (left, top),
// 3 (right, top).  For each (face or corner, m): active (a boundary value is
// imposed), refl (reflected ordinate), f (Fresnel coefficient of the
// governing face); exitance weight w (1 - f) cos for outgoing ordinates.
struct BoundaryTables {
  std::vector<int> face_refl, corner_refl;      // [4*M]
  std::vector<double> face_f, corner_f;         // [4*M]
  std::vector<unsigned char> face_act, corner_act;
  std::vector<double> wexit;                    // [4*M]
};
void boundary_tables(int M, double n_in, double n_out, BoundaryTables& bt);

// Transpose of the linear part of the boundary map (the source term is a
// constant): on a node of table tb (faces 0..3, corners 4..7 of bt),
// w[k] = sum_{q < 4} f[(tb M + k) 4 + q] ubar[src[(tb M + k) 4 + q]], with
// slot 0 the node's own value (kept where k is not imposed) and slots 1..3
// the imposed ordinates m whose reflection is k, weighted by their Fresnel
// coefficient; unused slots have f = 0.  Returns false if some k is the
// reflection of more than three imposed ordinates.
bool bc_transpose_tables(const BoundaryTables& bt, int M, std::vector<int>& src, std::vector<double>& f);

// Ring of boundary nodes: face 0 nodes j = 0..ny-1, then face 1 (j), face 2
// (i = 0..nx-1), face 3 (i); node positions and trapezoid weights.
void ring_geometry(int nx, int ny, double xmin, double xmax, double ymin, double ymax,
                   std::vector<double>& px, std::vector<double>& py,
                   std::vector<double>& weight);

}  // namespace rte_setup
