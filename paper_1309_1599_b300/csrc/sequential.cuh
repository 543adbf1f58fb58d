// Sequential overrelaxation sweep (App. A.1): the sites of a lattice are
// visited one at a time in the natural order i = x + L (y + L z), each
// reflected about the field of its neighbours' current values, so the update
// travels through the lattice as a wave.
//
// The sweep is executed exactly, in parallel, by hyperplanes: every
// neighbour that the natural order visits before a site has a smaller
// x + y + z (periodic wraps included: the wrapped neighbour of x = 0 is at
// x = L-1, visited later and further along x + y + z) and every later one a
// larger x + y + z, and two sites of one hyperplane x + y + z = tau are never
// neighbours.  So updating the hyperplanes tau = 0 .. 3L-3 in turn, each from
// the state left by the previous one, is the sequential sweep.
//
// A CTA owns one lattice group (V interleaved lattices), held in shared
// memory in natural site order [3][N][V] for the whole launch; the couplings
// are read from global memory.  The field is summed in the order of the
// other sweep kernels (+x, +y, +z and -x, -y, -z partial sums).
#pragma once
#include "kernels.cuh"

namespace hsg {

constexpr int kSeqThreads = 256;

struct SeqParams {
  BucketView b;
  int n_sweeps;
};

template <int V, int PREC>
__global__ void __launch_bounds__(kSeqThreads) k_sweep_or_seq(SeqParams p) {
  extern __shared__ __align__(16) float ssp[];  // [3][N][V], natural order
  const BucketView& b = p.b;
  const int L = b.L, N = b.N, LL = L * L;
  const int gi = blockIdx.x;                    // lattice group of the bucket
  const int sb = gi / b.G;
  float* gs = b.spins + static_cast<size_t>(gi) * 3 * N * V;
  const void* Jb = sample_bonds<PREC>(b.J, sb, N);
  const int plane = N * V;

  // global (parity-split rows) -> shared (natural order)
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
    const int c = q / N, i = q - c * N;
    const int x = i % L, row = i / L;
    const int src = site_of<true>(x, row, L);
#pragma unroll
    for (int v = 0; v < V; ++v) ssp[c * plane + i * V + v] = gs[static_cast<size_t>(c) * plane + src * V + v];
  }
  __syncthreads();

  for (int sweep = 0; sweep < p.n_sweeps; ++sweep) {
    for (int tau = 0; tau <= 3 * (L - 1); ++tau) {
      for (int j = threadIdx.x; j < LL; j += blockDim.x) {
        const int y = j % L, z = j / L;
        const int x = tau - y - z;
        if (x < 0 || x >= L) continue;
        const int row = y + L * z;
        const int xp = (x == L - 1) ? 0 : x + 1, xm = (x == 0) ? L - 1 : x - 1;
        const int yp = (y == L - 1) ? 0 : y + 1, ym = (y == 0) ? L - 1 : y - 1;
        const int zp = (z == L - 1) ? 0 : z + 1, zm = (z == 0) ? L - 1 : z - 1;
        const int i = x + L * row;
        // natural indices of the six neighbours
        const int n_xp = xp + L * row, n_xm = xm + L * row;
        const int n_yp = x + L * (yp + L * z), n_ym = x + L * (ym + L * z);
        const int n_zp = x + L * (y + L * zp), n_zm = x + L * (y + L * zm);
        // storage positions of the bonds: the site's own (+x, +y, +z) and
        // those of its -x, -y, -z neighbours
        const size_t pos = site_of<true>(x, row, L);
        const size_t pxm = site_of<true>(xm, row, L);
        const size_t pym = site_of<true>(x, ym + L * z, L);
        const size_t pzm = site_of<true>(x, y + L * zm, L);
        float hf[3][V], hb[3][V], h[3][V], j6[6], s[3][V];
        zero3<V>(hf);
        zero3<V>(hb);
        auto nb = [&](int n) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int v = 0; v < V; ++v) s[c][v] = ssp[c * plane + n * V + v];
        };
        load_bond<PREC>(Jb, pos, j6, b.D);                        nb(n_xp); add_bond<V>(j6, s, hf);
        load_bond<PREC>(Jb, N + pos, j6, b.D);                    nb(n_yp); add_bond<V>(j6, s, hf);
        load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + pos, j6, b.D); nb(n_zp); add_bond<V>(j6, s, hf);
        load_bond<PREC>(Jb, pxm, j6, b.D);                        nb(n_xm); add_bond<V>(j6, s, hb);
        load_bond<PREC>(Jb, N + pym, j6, b.D);                    nb(n_ym); add_bond<V>(j6, s, hb);
        load_bond<PREC>(Jb, 2 * static_cast<size_t>(N) + pzm, j6, b.D); nb(n_zm); add_bond<V>(j6, s, hb);
        combine_field<V>(hf, hb, h);
        nb(i);
        overrelax_v<V>(h, s);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int v = 0; v < V; ++v) ssp[c * plane + i * V + v] = s[c][v];
      }
      __syncthreads();
    }
  }

  // shared -> global
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
    const int c = q / N, i = q - c * N;
    const int x = i % L, row = i / L;
    const int dst = site_of<true>(x, row, L);
#pragma unroll
    for (int v = 0; v < V; ++v) gs[static_cast<size_t>(c) * plane + dst * V + v] = ssp[c * plane + i * V + v];
  }
}

}  // namespace hsg
