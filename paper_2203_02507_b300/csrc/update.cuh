// Fused per-LED update of one tile (one LED sub-aperture), on one CTA or on a
// cluster of C CTAs that share the work through distributed shared memory.
//
// Per update (alternating projection, Sec. 2.1; pupil correction of EPRY):
//   Phi  = O_box * P                  (box of m x m centred at c + s)
//   phi~ = IDFT_m(Phi)                (unnormalised; the (m/N)^2 / m^2 factor
//                                      cancels in phi~/|phi~|)
//   phi' = sqrt(I) phi~/|phi~|        (sqrt(I) where phi~ = 0)
//   Phi' = (N/m)^2 DFT_m(phi')
//   D    = Phi' - Phi
//   O_box += conj(P) D / max|P|^2,  dP = conj(O_box_old) D / max|O_box_old|^2
// Both maxima are reduced over the support inside the update.
// The box is taken in its centred order: transforming a centred spectrum as if
// it were in natural order multiplies the spatial field by (-1)^(x+y), which
// the amplitude step preserves and the forward transform undoes, so no shift
// is ever applied.
//
// Layout of the 2-D transform (m = A * B, both factors at most 16):
//   phase 1  rows of the support (R rows): IDFT along x  -> shared "inter" [R][m]
//   phase 2  every column: IDFT along y, amplitude step, DFT along y, keep R rows
//   phase 3  rows of the support: DFT along x, spectrum and pupil update
// Rows outside the support are zero before phase 1 and unused after phase 2,
// so only R x m values are ever stored.  Each 1-D transform of length m is run
// by TPT lanes of one warp in two register passes (radix A and radix B) with
// one exchange through a per-group shared scratch; phases are separated by
// a CTA (C = 1) or cluster (C > 1) barrier.  With C > 1 the columns of "inter"
// are split across the cluster: CTA q holds columns [q m/C, (q+1) m/C).
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <type_traits>

#include "aux_kernels.cuh"
#include "dft.cuh"
#include "update_args.h"

namespace cg = cooperative_groups;

namespace fpm {


// Swizzled position in "inter" (row length W, a multiple of 16) of local column p
// of stored row i, which holds box row y: the 4-bit XOR key h(y) ^ (p >> 4) moves
// p within its aligned block of 16 columns.  A warp touches inter in two
// patterns: TPT consecutive rows of 32 / TPT consecutive columns (the column
// phase), and TPT consecutive columns of 32 / TPT consecutive rows (the row
// phases).  8-byte accesses are served half a warp at a time, so each pattern is
// free of bank conflicts when the 16 lanes of a half warp meet 16 different
// bank pairs.  h(y) = y mod 16 does this for 16 lanes per transform; for 8,
// h(y) = (y & 6) | (y & 1) << 3 (the columns of a half warp differ in bit 0, its
// rows in bit 3); for 4, h(y) = 4 (y & 3) (columns in bits 0-1, rows in bits
// 2-3).  A lane that walks rows y = B a + b (B a multiple of 8) keeps a constant
// key.
template <int TPT>
__device__ __forceinline__ int inter_key(int y) {
  if constexpr (TPT >= 16) return y & 15;
  else if constexpr (TPT == 8) return (y & 6) | ((y & 1) << 3);
  else return (y & 3) << 2;
}
template <int TPT>
__device__ __forceinline__ int inter_swz(int y, int p) { return p ^ ((inter_key<TPT>(y) ^ (p >> 4)) & 15); }
template <int TPT>
__device__ __forceinline__ int inter_at(int i, int y, int p, int w) { return i * w + inter_swz<TPT>(y, p); }

// Accesses to a cluster CTA's shared memory through its 32-bit shared::cluster
// address (mapa), not through a generic pointer.
__device__ __forceinline__ uint32_t cluster_addr(const void *local_smem, int rank) {
  uint32_t r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local_smem)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// B consecutive image elements of one column (one lane's pixels in the column
// phase), fetched with 16-byte loads and kept packed until they are used.
template <typename Img, int B>
struct ImgCol {
  static_assert(B % 8 == 0, "a lane's pixels span whole 16-byte words");
  static constexpr int WORDS = (int)(B * sizeof(Img) / 4);
  unsigned w[WORDS];
  __device__ __forceinline__ void load(const Img *p) {
#pragma unroll
    for (int i = 0; i < WORDS / 4; ++i) {
      const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + i);
      w[4 * i] = v.x;
      w[4 * i + 1] = v.y;
      w[4 * i + 2] = v.z;
      w[4 * i + 3] = v.w;
    }
  }
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < WORDS; ++i) w[i] = 0u;
  }
  // pixel k as a float: a 16-bit value u is placed in the mantissa of 2^23
  // (one byte permute) and 2^23 subtracted, exact for every u < 2^23
  __device__ __forceinline__ float get(int k) const {
    if constexpr (sizeof(Img) == 2) {
      const unsigned bits = __byte_perm(w[k >> 1], 0x4B000000u, (k & 1) ? 0x7632u : 0x7610u);
      return __fadd_rn(__uint_as_float(bits), -8388608.0f);
    } else {
      return __uint_as_float(w[k]);
    }
  }
  // the measured counts of pixel k (intensity = counts / counts_per_unit),
  // negative values clamped to zero (16-bit counts are never negative)
  __device__ __forceinline__ float counts(int k) const {
    if constexpr (sizeof(Img) == 2) return get(k);
    else return fmaxf(get(k), 0.f);
  }
};

// PF_ = 1: a lane loads its next column's image pixels one column ahead;
// 0: at the start of the column (8 registers fewer for 16-bit images, 16 for float).
// PR_ = 1: a lane loads its next support row's spectrum and pupil values during
// the second pass of the current row (4 A registers more); 0: at the row's start.
// TG_ = 1: the twiddles are read from global memory (they stay in L1) instead of
// shared memory, 4 KB less shared memory per CTA at m = 256.
// DS_ = 1: the other CTAs' "inter" is accessed through 32-bit shared::cluster
// addresses (mapa); 0: through generic pointers (map_shared_rank), which leaves
// the register allocator more freedom where the update is inlined into a loop
// with state of its own (the persistent kernel).
// ZB_ > 0 (A = 16 only): the support lies in positions [ZB B, (A - ZB) B) of the
// box in both directions (band_fits), so the radix-A passes that take support
// samples skip their ZB zero blocks at each end, and those that give them
// compute only the blocks in the band (DftBand16); 0: every block.
template <int M_, int A_, int B_, int TPT_, int C_, int T_, int MINB_ = 1, int PF_ = 1, int PR_ = 0, int TG_ = 0,
          int DS_ = 1, int ZB_ = 0>
struct UpdateCfg {
  static constexpr int M = M_, A = A_, B = B_, TPT = TPT_, C = C_, T = T_, MINB = MINB_, PF = PF_, PR = PR_;
  static constexpr int TG = TG_, DS = DS_, ZB = ZB_;
  static_assert(ZB == 0 || (A == 16 && 2 * ZB < A), "band pruning needs the radix-16 first pass");
  static constexpr int W = M / C;          // columns of "inter" held by one CTA
  static constexpr int G = T / TPT;        // transforms in flight per CTA
  // exchange scratch of one group (complex values): the padded 2-D block, and for
  // groups narrower than 16 lanes at m <= 128 a little more, so that the groups
  // that share a warp start TPT banks apart (the groups' 8-byte accesses then
  // fill a wavefront instead of landing on the same banks)
  static constexpr int SCR0 = (B * (A + 1) > A * (B + 1)) ? B * (A + 1) : A * (B + 1);
  static constexpr int SCR = (TPT < 16 && M <= 128) ? SCR0 + ((TPT - SCR0 % 16) % 16 + 16) % 16 : SCR0;
  static constexpr int UA = (B + TPT - 1) / TPT;   // units of the radix-A passes per lane
  static constexpr int UB = (A + TPT - 1) / TPT;   // units of the radix-B passes per lane
  static_assert(A * B == M, "m = A * B");
  static_assert(A == image_split_a(M), "the tile images are laid out for the canonical split of m");
  static_assert(32 % TPT == 0 && T % 32 == 0, "groups must not straddle warps");
  static_assert(W % 16 == 0, "inter rows are swizzled in groups of 16");
  static_assert(T <= 512, "the normaliser holds one partial per warp in 16 slots");
  // shared memory in bytes for R support rows
  static size_t smem_bytes(int rows) {
    return ((size_t)rows * W + (size_t)G * SCR + (TG ? 0 : 2 * M)) * sizeof(float2) + 64 * sizeof(float);
  }
};

// The configuration Cfg with band pruning Z (kBandBlocks: for m = 256 and 128
// every support of the configs lies in the band).
template <class Cfg, int Z>
using WithBand = UpdateCfg<Cfg::M, Cfg::A, Cfg::B, Cfg::TPT, Cfg::C, Cfg::T, Cfg::MINB, Cfg::PF, Cfg::PR, Cfg::TG,
                           Cfg::DS, Z>;

// Whether block j of a radix-A pass over the support samples (positions
// B j + lane) can hold a nonzero sample / a needed output.
template <class Cfg>
__device__ __forceinline__ constexpr bool in_band(int j) {
  return Cfg::ZB == 0 || (j >= Cfg::ZB && j < Cfg::A - Cfg::ZB);
}

// The radix-A pass whose inputs are support samples (zero outside the band), and
// the one whose outputs are (only those in the band are needed).
template <class Cfg, int S>
__device__ __forceinline__ void dft_a_in(float2 *v) {
  if constexpr (Cfg::ZB > 0) DftBand16<S, Cfg::ZB, Cfg::A - 1 - Cfg::ZB, 0, 15>::run(v);
  else Dft<Cfg::A, S>::run(v);
}
template <class Cfg, int S>
__device__ __forceinline__ void dft_a_out(float2 *v) {
  if constexpr (Cfg::ZB > 0) DftBand16<S, 0, 15, Cfg::ZB, Cfg::A - 1 - Cfg::ZB>::run(v);
  else Dft<Cfg::A, S>::run(v);
}

// Twiddle i of a table: a shared-memory load, or a read-only global load (Cfg::TG).
template <class Cfg>
__device__ __forceinline__ float2 tw_at(const float2 *t, int i) {
  if constexpr (Cfg::TG) return __ldg(t + i);
  else return t[i];
}

// The transform twiddles of tile side M into the start of shared memory (the
// caller synchronises before run_update reads them).
template <class Cfg>
__device__ __forceinline__ void load_twiddles(const UpdateArgs &a, float2 *smem) {
  if constexpr (Cfg::TG) return;
  for (int i = threadIdx.x; i < Cfg::M; i += Cfg::T) {
    smem[i] = a.tw_inv[i];
    smem[Cfg::M + i] = a.tw_fwd[i];
  }
}

// No work at the hook point of run_update.
struct NoHook {
  __device__ __forceinline__ void operator()(int) const {}
};

// One update; all threads of all C CTAs of the cluster call this with the same item.
// Shared memory: [twiddles 2m (not with Cfg::TG)][normaliser partials][inter R x W][exchange scratch].
// load_tw = false keeps the twiddles of an earlier update with the same m.
// ordered_end = true: the closing cluster barrier also orders this update's global
// writes before whatever the cluster does next; false: the barrier only keeps the
// CTAs' shared memory alive until the cluster has read it (with a hook, its warp
// releases what the hook wrote into the CTAs' shared memory), and the kernel's
// end or a later cluster barrier orders the global writes (the persistent kernel
// counts an update done only after the next update's phase barriers).
// hook(0) and hook(1) run on one thread (cluster rank 0, the first lane of the
// last warp, whose groups have the fewest phase-3 rows): hook(0) before its
// phase-3 rows (for requests whose answers it needs only later), hook(1) after
// them and before the closing barrier, which publishes what it writes to shared
// memory.
template <class Cfg, typename Img, class Hook = NoHook>
__device__ __forceinline__ void run_update(const UpdateArgs &a, int4 item, float2 *smem, bool load_tw = true,
                                           bool ordered_end = true, const Hook &hook = Hook{}) {
  constexpr int M = Cfg::M, A = Cfg::A, B = Cfg::B, TPT = Cfg::TPT, C = Cfg::C, T = Cfg::T;
  constexpr int W = Cfg::W, G = Cfg::G, SCR = Cfg::SCR;
  const int rows = a.rows;
  const float2 *twi = Cfg::TG ? a.tw_inv : smem;
  const float2 *twf = Cfg::TG ? a.tw_fwd : smem + M;
  float2 *const tw_end = Cfg::TG ? smem : smem + 2 * M;
  float *red = reinterpret_cast<float *>(tw_end);
  float2 *inter = tw_end + 32;              // after 64 floats of partials
  float2 *scratch_all = inter + (size_t)rows * W;

  const int tid = threadIdx.x;
  const int g = tid / TPT, tl = tid % TPT;
  const unsigned lane = tid & 31;
  const unsigned gmask = (TPT == 32) ? 0xffffffffu : (((1u << TPT) - 1u) << (lane & ~(unsigned)(TPT - 1)));
  float2 *scr = scratch_all + g * SCR;

  int q = 0;
  float2 *inter_of[C];
  uint32_t inter_cl[C];                     // shared::cluster addresses of the CTAs' inter
  if constexpr (C > 1) {
    cg::cluster_group cl = cg::this_cluster();
    q = (int)cl.block_rank();
#pragma unroll
    for (int r = 0; r < C; ++r) {
      if constexpr (Cfg::DS) inter_cl[r] = cluster_addr(inter, r);
      else inter_of[r] = cl.map_shared_rank(inter, r);
    }
  } else {
    inter_of[0] = inter;
  }

  const int tile = item.x, led = item.y, slot = item.z;
  const int2 sh = a.shifts[(size_t)tile * a.n_leds + led];
  const int n = a.n;
  const int oy = n / 2 + sh.x - M / 2, ox = n / 2 + sh.y - M / 2;
  float2 *__restrict__ spec = a.spec + (size_t)tile * n * n + (size_t)oy * n + ox;   // box origin
  const size_t mm = (size_t)M * M;
  const float2 *__restrict__ pup = a.pup + (size_t)tile * mm;
  float2 *dp_out = a.dpup ? a.dpup + ((size_t)tile * a.slots + slot) * mm : nullptr;
  // this CTA's first column of the tile image (column-permuted layout)
  const Img *img = reinterpret_cast<const Img *>(a.images) + tile_image_offset(tile, led, a.n_leds, M) +
                   (size_t)q * W * M;

  // rows of the support handled by this CTA in phases 1 and 3
  const int rpc = (rows + C - 1) / C;
  const int r0 = q * rpc, r1 = min(rows, r0 + rpc);

  if (load_tw) load_twiddles<Cfg>(a, smem);
  __syncthreads();

  // ---- phase 1: IDFT along x of every support row -------------------------
  // A lane's spectrum and pupil values of its next row are loaded while the
  // second pass of the current row runs (Cfg::PR), so their latency overlaps
  // that pass instead of opening every row.
  float omax = 0.f, pmax = 0.f;
  float2 ov1[Cfg::UA][A], pv1[Cfg::UA][A];
  auto load_row = [&](int i) {
    const int by = a.y_lo + i;
    const int2 ch = a.chords[by];
    const float2 *__restrict__ srow = spec + (size_t)by * n;
    const float2 *__restrict__ prow = pup + (size_t)by * M;
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int b = tl + u * TPT;
#pragma unroll
      for (int aa = 0; aa < A; ++aa) {
        const int x = B * aa + b;
        const bool in = in_band<Cfg>(aa) && b < B && x >= ch.x && x <= ch.y;
        ov1[u][aa] = in ? srow[x] : make_float2(0.f, 0.f);
        pv1[u][aa] = in ? prow[x] : make_float2(0.f, 0.f);
      }
    }
  };
  if (Cfg::PR && r0 + g < r1) load_row(r0 + g);
  for (int i = r0 + g; i < r1; i += G) {
    const int by = a.y_lo + i;
    // the group's next row into L2 while this one is worked on: lane l asks for
    // the l-th 16-sample piece of its spectrum and pupil rows where it meets the
    // support chord (no registers held)
    if (i + G < r1 && tl * 16 < M) {
      const int2 nc = a.chords[by + G];
      if (tl * 16 + 15 >= nc.x && tl * 16 <= nc.y) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(spec + (size_t)(by + G) * n + tl * 16));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(pup + (size_t)(by + G) * M + tl * 16));
      }
    }
    if constexpr (!Cfg::PR) load_row(i);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int b = tl + u * TPT;
      if (b < B) {
        float2 v[A];
#pragma unroll
        for (int aa = 0; aa < A; ++aa) {
          v[aa] = make_float2(0.f, 0.f);
          if (!in_band<Cfg>(aa)) continue;        // zero outside the band
          omax = fmaxf(omax, cabs2(ov1[u][aa]));
          pmax = fmaxf(pmax, cabs2(pv1[u][aa]));
          v[aa] = cmul(ov1[u][aa], pv1[u][aa]);
        }
        dft_a_in<Cfg, 1>(v);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
          const float2 w = tw_at<Cfg>(twi, k1 * B + b);
          scr[b * (A + 1) + k1] = (k1 == 0) ? v[0] : cmul(v[k1], w);
        }
      }
    }
    __syncwarp(gmask);
    if constexpr (Cfg::PR) {
      if (i + G < r1) load_row(i + G);
    }
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
        float2 v[B];
#pragma unroll
        for (int bb = 0; bb < B; ++bb) v[bb] = scr[bb * (A + 1) + k1];
        Dft<B, 1>::run(v);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          const int x = k1 + A * k2;
          const int owner = (C > 1) ? x / W : 0;
          const int p = (C > 1) ? x - owner * W : x;
          if constexpr (C > 1 && Cfg::DS) st_cluster(inter_cl[owner] + 8u * (uint32_t)inter_at<TPT>(i, by, p, W), v[k2]);
          else inter_of[owner][inter_at<TPT>(i, by, p, W)] = v[k2];
        }
      }
    }
    __syncwarp(gmask);
  }
  // normalisers: max |O_box_old|^2 and max |P|^2 over the support, over the whole cluster
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, o));
    pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
  }
  if (lane == 0) {
    red[tid >> 5] = omax;
    red[16 + (tid >> 5)] = pmax;
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }
  // the last warp (whose groups have the fewest columns in phase 2) combines
  // the cluster's partials while the others start phase 2; phase 3 reads the
  // result after the phase 2 barrier
  if (tid >= T - 32) {
    const int l = tid - (T - 32), wi = l & 15;
    float v = (wi < T / 32) ? red[l] : 0.f;            // lanes 0-15: |O|^2, 16-31: |P|^2
    if constexpr (C > 1) {
      cg::cluster_group cl = cg::this_cluster();
      for (int r = 0; r < C; ++r)
        if (r != q && wi < T / 32) v = fmaxf(v, cl.map_shared_rank(red, r)[l]);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) red[32] = v;
    if (l == 16) red[33] = v;
  }

  // ---- phase 2: columns: IDFT along y, amplitude step, DFT along y ---------
  const int y_lo = a.y_lo, y_hi = a.y_lo + rows - 1;
  // per lane: which rows y = B a + b (first pass) and y = kk + B k2 (last pass) are stored
  unsigned in_mask[Cfg::UA], out_mask[Cfg::UA];
#pragma unroll
  for (int u = 0; u < Cfg::UA; ++u) {
    const int b = tl + u * TPT;
    in_mask[u] = 0;
    out_mask[u] = 0;
#pragma unroll
    for (int aa = 0; aa < A; ++aa) {
      const int y = B * aa + b;
      if (b < B && y >= y_lo && y <= y_hi) in_mask[u] |= 1u << aa;
    }
#pragma unroll
    for (int k2 = 0; k2 < A; ++k2) {
      const int y = b + B * k2;
      if (b < B && y >= y_lo && y <= y_hi) out_mask[u] |= 1u << k2;
    }
  }
  // measured pixels of this lane's rows y = k1 + A k2 (B contiguous elements)
  ImgCol<Img, B> meas[Cfg::UB];
  auto fetch = [&](int col, ImgCol<Img, B> (&dst)[Cfg::UB]) {
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A && col < W) dst[u].load(img + (size_t)col * M + k1 * B);
      else dst[u].zero();
    }
  };
  if constexpr (Cfg::PF) fetch(g, meas);
  for (int c = g; c < W; c += G) {
    ImgCol<Img, B> next[Cfg::PF ? Cfg::UB : 1];
    if constexpr (Cfg::PF) fetch(c + G, next);
    else fetch(c, meas);                   // consumed after the first pass
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int b = tl + u * TPT;
      if (b < B) {
        float2 v[A];
        const float2 *col_base = inter + (b - y_lo) * W;   // row y = B aa + b is stored at i = y - y_lo
#pragma unroll
        for (int aa = 0; aa < A; ++aa)
          v[aa] = (in_band<Cfg>(aa) && ((in_mask[u] >> aa) & 1u)) ? col_base[aa * B * W + inter_swz<TPT>(B * aa + b, c)]
                                                                 : make_float2(0.f, 0.f);
        dft_a_in<Cfg, 1>(v);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) scr[b * (A + 1) + k1] = (k1 == 0) ? v[0] : cmul(v[k1], tw_at<Cfg>(twi, k1 * B + b));
      }
    }
    __syncwarp(gmask);
    float2 keep[Cfg::UB][B];
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
        float2 *v = keep[u];
#pragma unroll
        for (int bb = 0; bb < B; ++bb) v[bb] = scr[bb * (A + 1) + k1];
        Dft<B, 1>::run(v);
        // amplitude step at y = k1 + A k2, without branches, in count units (the
        // factor sqrt(1/counts_per_unit) joins the forward scale in phase 3):
        // sqrt(c) / |phi~| = c / sqrt(c |phi~|^2) with the hardware reciprocal
        // square root (a couple of ulp; a Newton-Raphson refinement cost 2% of the
        // update and moved the parity errors by less than their float32 floor).
        // x = c |phi~|^2 + FLT_MIN (one fused multiply-add; the FLT_MIN changes no
        // value of x above 2^-102 and keeps x > 0), so c = 0 gives 0 * (finite r)
        // = 0 with no select.  Where phi~ = 0 (rare: the smallest |phi~|^2 of the
        // lane is 0) the result is 0, and every pixel left at 0 takes sqrt(c)
        // afterwards (which is 0 again where c = 0).
        float m2min = 1.f;
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
          const float cn = meas[u].counts(k2);
          const float2 f = v[k2];
          const float m2 = cabs2(f);
          m2min = fminf(m2min, m2);
          const float x = __fmaf_rn(cn, m2, 1.17549435e-38f);
          const float r = rsqrtf(x);
          v[k2] = cscale(f, __fmul_rn(cn, r));
        }
        if (m2min == 0.f) {
#pragma unroll
          for (int k2 = 0; k2 < B; ++k2)
            if (v[k2].x == 0.f && v[k2].y == 0.f) v[k2] = make_float2(sqrtf(meas[u].counts(k2)), 0.f);
        }
        // forward DFT, first pass of the B x A split: unit b' = k1, over a' = k2
        Dft<B, -1>::run(v);
      }
    }
    __syncwarp(gmask);   // everyone has read scr
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int k1 = tl + u * TPT;
      if (k1 < A) {
#pragma unroll
        for (int kk = 0; kk < B; ++kk)
          scr[k1 * (B + 1) + kk] = (kk == 0) ? keep[u][0] : cmul(keep[u][kk], tw_at<Cfg>(twf, kk * A + k1));
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;   // k1' in [0, B)
      if (kk < B) {
        float2 v[A];
#pragma unroll
        for (int bb = 0; bb < A; ++bb) v[bb] = scr[bb * (B + 1) + kk];
        dft_a_out<Cfg, -1>(v);
        float2 *col_base = inter + (kk - y_lo) * W;
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2)
          if (in_band<Cfg>(k2) && ((out_mask[u] >> k2) & 1u)) col_base[k2 * B * W + inter_swz<TPT>(kk + B * k2, c)] = v[k2];
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u)
      if constexpr (Cfg::PF) meas[u] = next[u];
  }
  if constexpr (C > 1) {
    cg::this_cluster().sync();
  } else {
    __syncthreads();
  }

  const float onorm = red[32], pn = red[33];
  const float inv_on = (onorm > 0.f) ? 1.f / onorm : 0.f;
  const float inv_pn = 1.f / pn;
  // (N/m)^2 times the count-unit factor of the amplitude step, and the
  // normalisers, as pairs for the packed FP32x2 products
  const float fs = __fmul_rn(a.scale, sqrtf(a.inv_counts));
  const float2 fs2 = make_float2(fs, fs);

  // ---- phase 3: DFT along x of the support rows, then the updates ----------
  constexpr bool kHook = !std::is_same<Hook, NoHook>::value;
  if constexpr (kHook) {
    if (q == 0 && tid == T - 32) hook(0);
  }
  for (int i = r0 + g; i < r1; i += G) {
    const int by = a.y_lo + i;
    const int2 ch = a.chords[by];
    float2 *__restrict__ srow = spec + (size_t)by * n;
    const float2 *__restrict__ prow = pup + (size_t)by * M;
    // O_box_old and P at this lane's outputs x = kk + B k2, fetched before the transform
    float2 ov[Cfg::UA][A], pv[Cfg::UA][A];
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;
#pragma unroll
      for (int k2 = 0; k2 < A; ++k2) {
        const int x = kk + B * k2;
        const bool in = in_band<Cfg>(k2) && kk < B && x >= ch.x && x <= ch.y;
        ov[u][k2] = in ? srow[x] : make_float2(0.f, 0.f);
        pv[u][k2] = in ? prow[x] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < Cfg::UB; ++u) {
      const int b2 = tl + u * TPT;   // b' in [0, A)
      if (b2 < A) {
        float2 v[B];
#pragma unroll
        for (int aa = 0; aa < B; ++aa) {
          const int x = A * aa + b2;
          const int owner = (C > 1) ? x / W : 0;
          const int p = (C > 1) ? x - owner * W : x;
          if constexpr (C > 1 && Cfg::DS) v[aa] = ld_cluster(inter_cl[owner] + 8u * (uint32_t)inter_at<TPT>(i, by, p, W));
          else v[aa] = inter_of[owner][inter_at<TPT>(i, by, p, W)];
        }
        Dft<B, -1>::run(v);
#pragma unroll
        for (int kk = 0; kk < B; ++kk) scr[b2 * (B + 1) + kk] = (kk == 0) ? v[0] : cmul(v[kk], tw_at<Cfg>(twf, kk * A + b2));
      }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int u = 0; u < Cfg::UA; ++u) {
      const int kk = tl + u * TPT;
      if (kk < B) {
        float2 v[A];
#pragma unroll
        for (int bb = 0; bb < A; ++bb) v[bb] = scr[bb * (B + 1) + kk];
        dft_a_out<Cfg, -1>(v);
#pragma unroll
        for (int k2 = 0; k2 < A; ++k2) {
          const int x = kk + B * k2;
          if (in_band<Cfg>(k2) && x >= ch.x && x <= ch.y) {
            const float2 o = ov[u][k2];
            const float2 p = pv[u][k2];
            // -Phi = -(O P), then D = Phi' - Phi as one packed fused multiply-add
            const float2 nphi = make_float2(__fmaf_rn(o.y, p.y, -__fmul_rn(o.x, p.x)),
                                            __fmaf_rn(-o.x, p.y, -__fmul_rn(o.y, p.x)));
            const float2 d = __ffma2_rn(v[k2], fs2, nphi);
            const float2 pc = cmulc(d, p);        // D * conj(P)
            srow[x] = make_float2(__fmaf_rn(pc.x, inv_pn, o.x), __fmaf_rn(pc.y, inv_pn, o.y));
            if (dp_out) {
              const float2 oc = cmulc(d, o);      // D * conj(O_old)
              dp_out[(size_t)by * M + x] = cscale(oc, inv_on);
            }
          }
        }
      }
    }
    __syncwarp(gmask);
  }
  if constexpr (kHook) {
    if (q == 0 && tid == T - 32) hook(1);
    __syncwarp();
  }
  // keep this CTA's shared memory alive until the cluster is done reading it
  if constexpr (C > 1) {
    if (ordered_end) {
      cg::this_cluster().sync();
    } else if (kHook && q == 0 && tid >= T - 32) {
      // the hook's warp releases what the hook wrote into the CTAs' shared memory
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
      // relaxed arrive: no wait for this thread's global stores to drain
      asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
    }
  }
}

template <class Cfg, typename Img>
__global__ void __launch_bounds__(Cfg::T, Cfg::MINB) update_kernel(const __grid_constant__ UpdateArgs a, long long item0) {
  extern __shared__ float4 smem_raw[];
  const int4 item = a.items[item0 + blockIdx.x / Cfg::C];
  run_update<Cfg, Img>(a, item, reinterpret_cast<float2 *>(smem_raw), true, false);
}

}  // namespace fpm
