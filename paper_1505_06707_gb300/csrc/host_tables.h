// Host FP64 table construction (see tables.cpp).
#pragma once
#include <complex>
#include <vector>

#include "soft.h"

namespace soft {

using cd = std::complex<double>;

struct ContourFn {
    int kind;
    double R0, rmax, theta, alpha;
    double e_cap, kmin;           // comparison absorbers (kinds SOFT_ABSORB_*)
    ContourFn(int kind, double R0, double rmax, double theta, double alpha, double e_cap = 2.0,
              double kmin = 0.25);
    bool q(double x, cd* out) const;
    cd inv_q(double x) const;
    cd z(double x) const;
    cd absorber(double x) const;  // U_a(x); 0 for the contours
};

// One grid axis: grid, momenta, contour and the periodic tridiagonal C.
struct Axis1D {
    int n = 0;
    double a = 0, b = 0, h = 0, tau = 0;
    std::vector<double> x, k;
    std::vector<cd> q, z;
    std::vector<cd> Cs, Cd, Cu;   // C[j][j-1], C[j][j], C[j][j+1] (indices mod n)
};

void build_axis(Axis1D& A, int n, double a, double b, const ContourFn& cf, double tau);
int find_block(const Axis1D& A, int* blk0, int* nb);
int strip_factor(const Axis1D& A, int blk0, int nb, std::vector<cd>& mf, std::vector<cd>& mb,
                 std::vector<cd>& g, double* check_err);
std::vector<int> dif_output_order(int logn, int logrm);
std::vector<cd> pass_twiddles(int logn, int logrm);
std::vector<cd> pass_twiddles_full(int logn, int logrm, int full_maxs);
cd soft_coulomb(const cd* z, int nd, double a2, double Z);

}  // namespace soft
