// Preconditioner tables of Sec. III (see band.cpp).
#pragma once
#include <utility>
#include <vector>

#include "host_tables.h"

namespace soft {

struct BandAxis {
    int n = 0;
    std::vector<cd> lam;          // lambda of each natural index nu
    std::vector<int> start;       // first index of nu's band
    std::vector<int> width;       // width of nu's band
    std::vector<int> off;         // offset of row nu in xf / xb
    std::vector<cd> xf;           // X[nu][m] e^{i k_m x0}/sqrt N, m over the band
    std::vector<cd> xb;           // X[m'][nu] e^{-i k_nu x0}/sqrt N: output nu, input m' over the band
};

std::vector<std::pair<int, int>> band_split(int n, int nbw);
int eig_complex_symmetric(int n, const std::vector<cd>& K, std::vector<cd>& lam,
                          std::vector<cd>& V, double* resid, double* orth);
int build_band_axis(const Axis1D& A, int nbw, bool simple, BandAxis& out, double* check);

}  // namespace soft
