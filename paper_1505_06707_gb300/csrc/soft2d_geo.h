// Geometry and table pointers of a 2D plan, passed by value to the 2D kernels.
#pragma once

namespace soft {

struct Geo2D {              // passed by value to every 2D kernel
    const void* Wx;         // pass twiddles of the row FFT (length nx)
    const void* Wy;         // pass twiddles of the column FFT (length ny)
    const void* TVh;        // e^{-iU tau/2}, [ny][nx] (minus 1, float2, for complex64)
    const void* cnx;        // x-strip LU (mf, mb, g) for the row pass
    const void* cny;        // y-strip LU (mf, mb, g) for the y-block pass
    int nx, ny;
    int nbx, blk0x;         // x-strip block (same for every row)
    int nby, blk0y;         // y-strip block (same for every column)
};

}  // namespace soft
