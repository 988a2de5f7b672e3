// Geometry and table pointers of a 2D or 3D plan, passed by value to the
// pass kernels.
#pragma once
#include <cstdint>

namespace soft {

struct Geo2D {              // passed by value to every 2D kernel
    const void* Wx;         // pass twiddles of the row FFT (length nx)
    const void* Wy;         // pass twiddles of the column FFT (length ny)
    const void* TVh;        // e^{-iU tau/2}, [ny][nx] (minus 1, float2, for complex64)
    const void* cnx;        // x-strip LU (mf, mb, g) for the row pass
    const void* cny;        // y-strip LU (mf, mb, g) for the column pass
    int nx, ny;             // row length; number of rows (3D: ny nz)
    int nbx, blk0x;         // x-strip block (same for every row)
    int nby, blk0y;         // y-strip block (same for every column)
    // v2 = 1: the row pass applies the second V/2 to the rows r outside the
    // y-strip block and outside the z-strip block, y = r mod ny1 and
    // z = r / ny1 (2D: ny1 = ny, no z block)
    int v2, ny1, nz1, nbz1, blk0z1;
};

// Lines along a strided axis: element i of line c of plane p sits at
// p plane + i ld + c, c < ld (2D columns: ld = nx, one plane; 3D y lines:
// ld = nx, plane = nx ny, nz planes; 3D z lines: ld = nx ny, one plane).
struct LineGeo {
    const void* W;          // pass twiddles of the line FFT
    int64_t ld, plane;
    const void* cn;         // strip CN LU (mf, mb, g) along the lines (COL_CVK)
    const void* tv;         // e^{-iU tau/2}, laid out as the state (COL_CVK)
    int nb, blk0;           // strip block along the lines (COL_CVK)
    // COL_CVK: with sel_div > 0 only lines whose (c / sel_div) mod sel_n lies
    // in the cyclic block sel_blk0 .. + sel_nb take V/2 off the strip block
    // (the row pass applied it on the others)
    int64_t sel_div;
    int sel_n, sel_nb, sel_blk0;
};

// The strip CN along a strided axis: the cyclic block blk0 .. blk0 + nb - 1
// (mod n) of every line, lines laid out as in LineGeo.
struct CnGeo {
    const void* cn;         // LU (mf, mb, g) of the block
    int nb, blk0, n;
    int64_t ld, plane;
};

}  // namespace soft
