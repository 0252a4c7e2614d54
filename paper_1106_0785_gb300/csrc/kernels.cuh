// kernels.cuh - device layout and kernel launchers shared by the C ABI.
//
// Device layout of one state buffer (private to the library): 16 planes,
// each (ny + 2) rows of `pitch` elements.  Node (i, j) of the grid sits at
// row j + 1 and column i + xoff; row 0 / ny + 1 and columns xoff - 1 /
// xoff + nx are the one-node ghost layer.  xoff = 128 bytes / element size,
// so every interior row starts on a 128-byte boundary, and the TMA box of a
// tile, which starts 4 elements left of the tile, starts on a 16-byte one.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "physics.cuh"

namespace mrtlb {

enum : int { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_WALL = 2 };

// Bits of the device error word.
enum : int { ERRBIT_NONPHYSICAL = 1, ERRBIT_TIMEOUT = 2 };

struct Layout {
  int nx, ny;
  int pitch;          // elements per padded row
  int xoff;           // column of interior node i = 0
  long long plane;    // elements per plane = (ny + 2) * pitch
  int i0, i1, j0, j1; // advanced (non-wall) nodes: [i0, i1) x [j0, j1)
  int bc[4];          // -x, +x, -y, +y (BC_*)
  __host__ __device__ long long node(int i, int j) const {
    return (long long)(j + 1) * pitch + (i + xoff);
  }
};

struct Walls {
  double ux[4], uy[4], T[4];  // per side
};

template <typename R>
void launch_step_plain(const R* fin, R* fout, const Layout& L, const Coef<R>& c, int* err,
                       cudaStream_t st);
template <typename R>
void launch_bc(R* f, const Layout& L, const Coef<double>& c64, const Walls& w, cudaStream_t st);
template <typename R>
void launch_pack(const R* dense, R* padded, const Layout& L, cudaStream_t st);
template <typename R>
void launch_unpack(const R* padded, R* dense, const Layout& L, cudaStream_t st);
template <typename R>
void launch_init_eq(const double* rho, const double* ux, const double* uy, const double* T,
                    R* f, const Layout& L, const Coef<double>& c64, cudaStream_t st);
template <typename R>
void launch_macros(const R* f, double* rho, double* ux, double* uy, double* T, const Layout& L,
                   cudaStream_t st);
// acc: 4 FP64 sums + 1 max (as the bit pattern of a non-negative double);
// Tprev: [ny][nx] FP64 temperatures of the previous call (updated in place)
template <typename R>
void launch_reduce(const R* f, double* acc, double* Tprev, int have_prev, const Layout& L,
                   cudaStream_t st);

}  // namespace mrtlb
