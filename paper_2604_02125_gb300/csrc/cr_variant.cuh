// cr_variant.cuh -- launchers of one (system, degree, precision) variant.
#pragma once
#include "cr_internal.h"
#include "crkfr_volume_lanes.cuh"

#include <algorithm>

namespace crk {

template <typename R> struct PP;
template <> struct PP<double> {
  static const PhysParams<double>& get(const LaunchCtx& c) { return c.pp64; }
  static const RefTab<double>& tab(const LaunchCtx& c) { return c.tb64; }
};
template <> struct PP<float> {
  static const PhysParams<float>& get(const LaunchCtx& c) { return c.pp32; }
  static const RefTab<float>& tab(const LaunchCtx& c) { return c.tb32; }
};

template <typename R> struct PPB;
template <> struct PPB<double> {
  static const PhysParams<double>& get(const BatchLaunch& b) { return b.pp64; }
  static const RefTab<double>& tab(const BatchLaunch& b) { return b.tb64; }
};
template <> struct PPB<float> {
  static const PhysParams<float>& get(const BatchLaunch& b) { return b.pp32; }
  static const RefTab<float>& tab(const BatchLaunch& b) { return b.tb32; }
};

template <class EQ, int N, typename R>
struct Variant {
  using L = VolLayout<EQ, N, R>;
  using LL = LaneLayout<EQ, N, R>;
  using PL = PersistLayout<EQ, N, R>;
  static constexpr bool kLanes = PL::fits();
  static size_t vol_smem(int epb) { return kLanes ? PL::bytes() : (size_t)epb * L::bytes_per_elem(); }
  // resident CTAs per SM of the persistent volume kernel (computed once)
  static int vol_occupancy() {
    static int occ = -1;
    if (occ < 0) {
      int nb = 0;
      if constexpr (kLanes) {
        cudaFuncSetAttribute(k_volume_lanes<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_volume_lanes<EQ, N, R>, LL::THREADS, PL::bytes());
      }
      occ = nb > 0 ? nb : 1;
    }
    return occ;
  }
  static cudaError_t volume(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (kLanes) {
      const long long ntiles = (c.ma.E + 31) / 32;
      const long long grid = std::min(ntiles, (long long)c.sms * vol_occupancy());
      k_volume_lanes<EQ, N, R><<<(unsigned)grid, LL::THREADS, PL::bytes(), s>>>(
          c.u, (R*)c.rbar, (R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot);
    } else {
      const long long grid = (c.ma.E + c.epb - 1) / c.epb;
      const int threads = c.epb * L::NF;
      const size_t smem = (size_t)c.epb * L::bytes_per_elem();
      k_volume_tile<EQ, N, R><<<(unsigned)grid, threads, smem, s>>>(c.u, (R*)c.rbar, (R*)c.trace, c.st, c.ma,
                                                                    PP<R>::get(c), PP<R>::tab(c), c.slot);
    }
    return cudaGetLastError();
  }
  static cudaError_t volume_stage(const LaunchCtx& c, cudaStream_t s, const double* u_in, int first) {
    if constexpr (kLanes) {
      const long long ntiles = (c.ma.E + 31) / 32;
      const long long grid = std::min(ntiles, (long long)c.sms * vol_stage_occupancy());
      k_volume_lanes_stage<EQ, N, R><<<(unsigned)grid, LL::THREADS, PL::bytes(), s>>>(
          u_in, (R*)c.rbar, (R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot, first);
    } else {
      const long long grid = (c.ma.E + c.epb - 1) / c.epb;
      const int threads = c.epb * L::NF;
      const size_t smem = (size_t)c.epb * L::bytes_per_elem();
      k_volume_tile_stage<EQ, N, R><<<(unsigned)grid, threads, smem, s>>>(
          u_in, (R*)c.rbar, (R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot, first);
    }
    return cudaGetLastError();
  }
  static int vol_stage_occupancy() {
    static int occ = -1;
    if (occ < 0) {
      int nb = 0;
      if constexpr (kLanes) {
        cudaFuncSetAttribute(k_volume_lanes_stage<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)PL::bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_volume_lanes_stage<EQ, N, R>, LL::THREADS, PL::bytes());
      }
      occ = nb > 0 ? nb : 1;
    }
    return occ;
  }
  using FL = FaceLaneLayout<EQ, N, R>;
  static constexpr bool kFaceLanes = FL::fits();
  static cudaError_t face_stage(const LaunchCtx& c, cudaStream_t s, int j, int ns) {
    const RkStage<R> rk{(R*)c.kbuf, j == ns - 1 ? c.u : c.ustage, j, ns};
    if constexpr (kFaceLanes) {
      const unsigned grid = (unsigned)((c.ma.E + 31) / 32);
      k_face_stage_lanes<EQ, N, R><<<grid, FL::THREADS, FL::bytes(), s>>>(
          c.u, (const R*)c.rbar, (const R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot, rk);
    } else {
      const long long total = c.ma.E * L::NP;
      const unsigned grid = (unsigned)((total + 255) / 256);
      k_face_stage<EQ, N, R><<<grid, 256, 0, s>>>(c.u, (const R*)c.rbar, (const R*)c.trace, c.st, c.ma,
                                                   PP<R>::get(c), PP<R>::tab(c), c.slot, rk);
    }
    return cudaGetLastError();
  }
  static constexpr bool kBatched = EQ::DIM == 2 && !EQ::NC && kLanes && kFaceLanes;
  static cudaError_t face_update(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (kFaceLanes) {
      const unsigned grid = (unsigned)((c.ma.E + 31) / 32);
      k_face_update_lanes<EQ, N, R><<<grid, FL::THREADS, FL::bytes(), s>>>(
          c.u, (const R*)c.rbar, (const R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot);
    } else {
      const long long total = c.ma.E * L::NP;
      const unsigned grid = (unsigned)((total + 255) / 256);
      k_face_update<EQ, N, R><<<grid, 256, 0, s>>>(c.u, (const R*)c.rbar, (const R*)c.trace, c.st, c.ma,
                                                    PP<R>::get(c), PP<R>::tab(c), c.slot);
    }
    return cudaGetLastError();
  }
  static constexpr bool kVolInd = kLanes && !EQ::NC && sizeof(R) == 4;
  static cudaError_t volume_ind(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (kVolInd) {
      static int occ = -1;
      if (occ < 0) {
        int nb = 0;
        cudaFuncSetAttribute(k_volume_lanes_ind<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)PL::bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_volume_lanes_ind<EQ, N, R>, LL::THREADS, PL::bytes());
        occ = nb > 0 ? nb : 1;
      }
      const long long ntiles = (c.ma.E + 31) / 32;
      const long long grid = std::min(ntiles, (long long)c.sms * occ);
      k_volume_lanes_ind<EQ, N, R><<<(unsigned)grid, LL::THREADS, PL::bytes(), s>>>(
          c.u, (R*)c.rbar, (R*)c.trace, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c), c.slot, c.araw, c.tcount, c.lt);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t alpha_smooth(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (!EQ::NC) {
      if constexpr (kVolInd)
        k_alpha_fix<EQ, N><<<(unsigned)((c.ma.E + 127) / 128), 128, 0, s>>>(c.u, c.araw, c.ma, c.lt);
      k_alpha_smooth<EQ::DIM><<<(unsigned)((c.ma.E + 255) / 256), 256, 0, s>>>(c.araw, c.alpha, c.touched, c.tlist,
                                                                              c.tcount, c.ma);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t alpha(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (!EQ::NC) {
      constexpr int T = AlphaRawLayout<EQ, N, R>::THREADS;
      const unsigned grid = (unsigned)((c.ma.E + T - 1) / T);
      k_alpha_raw<EQ, N, R><<<grid, T, 0, s>>>(c.u, c.araw, c.tcount, c.ma, c.lt);
      k_alpha_smooth<EQ::DIM><<<(unsigned)((c.ma.E + 255) / 256), 256, 0, s>>>(c.araw, c.alpha, c.touched, c.tlist,
                                                                              c.tcount, c.ma);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  // the limited face / update part: the lane kernel for the elements the
  // limiter does not touch, the per-node limited kernel for the others (all
  // elements where the lane layout does not fit)
  static cudaError_t face_limited(const LaunchCtx& c, cudaStream_t s) {
    if constexpr (!EQ::NC) {
      if constexpr (kFaceLanes) {
        const unsigned tiles = (unsigned)((c.ma.E + 31) / 32);
        k_face_update_lanes_clean<EQ, N, R><<<tiles, FL::THREADS, FL::bytes(), s>>>(
            c.u, c.u_next, (const R*)c.rbar, (const R*)c.trace, c.touched, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c),
            c.slot);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      // over the touched elements' nodes (their number is known on the device
      // only: a grid of four CTAs per SM strides over them), else over all nodes
      const long long total = c.ma.E * L::NP;
      const unsigned grid = (unsigned)std::min((total + 255) / 256, kFaceLanes ? 4LL * c.sms : (total + 255) / 256);
      k_face_update_limited<EQ, N, R><<<grid, 256, 0, s>>>(c.u, c.u_next, (const R*)c.rbar, (const R*)c.trace, c.alpha,
                                                           c.tlist, c.tcount, c.st, c.ma, PP<R>::get(c), PP<R>::tab(c),
                                                           c.lt, c.slot, kFaceLanes ? 1 : 0);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  using FU = FusedLayout<EQ, N, R>;
  static constexpr bool kFused = FU::fits() && !EQ::NC;
  static int fused_occupancy() {
    static int occ = -1;
    if (occ < 0) {
      int nb = 0;
      if constexpr (kFused) {
        cudaFuncSetAttribute(k_step_fused<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FU::bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_fused<EQ, N, R>, LL::THREADS, FU::bytes());
      }
      occ = nb;
    }
    return occ;
  }
  static cudaError_t step_fused(const LaunchCtx& c, cudaStream_t s, int phase) {
    if constexpr (kFused) {
      const int occ = fused_occupancy();
      if (occ < 1) return cudaErrorInvalidConfiguration;
      const long long ntiles = (c.ma.E + 31) / 32;
      // cooperative: every CTA resident, so the bounded readiness waits end
      const long long grid = std::min(ntiles, (long long)c.sms * occ);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)grid);
      cfg.blockDim = dim3(LL::THREADS);
      cfg.dynamicSmemBytes = FU::bytes();
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_step_fused<EQ, N, R>, c.u, (R*)c.rbar, (R*)c.trace, c.st, c.flags, c.ma,
                                PP<R>::get(c), PP<R>::tab(c), phase);
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t lambda(const LaunchCtx& c, cudaStream_t s) {
    const long long total = c.ma.E * L::NP;
    const unsigned grid = (unsigned)((total + 255) / 256);
    k_lambda<EQ, N, R><<<grid, 256, 0, s>>>(c.u, c.st, c.ma, c.slot);
    return cudaGetLastError();
  }
  static cudaError_t totals(const LaunchCtx& c, cudaStream_t s) {
    const long long total = c.ma.E * L::NP;
    const unsigned grid = (unsigned)((total + 255) / 256);
    k_totals<EQ, N><<<grid, 256, 0, s>>>(c.u, c.totals_part, c.ma, c.tb64);
    return cudaGetLastError();
  }
  static cudaError_t set_smem(size_t bytes) {
    if constexpr (kFaceLanes) {
      cudaError_t e = cudaFuncSetAttribute(k_face_update_lanes<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FL::bytes());
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_face_stage_lanes<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)FL::bytes());
      if (e != cudaSuccess) return e;
      if constexpr (!EQ::NC) {
        e = cudaFuncSetAttribute(k_face_update_lanes_clean<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FL::bytes());
        if (e != cudaSuccess) return e;
      }
      if constexpr (kBatched) {
        e = cudaFuncSetAttribute(k_face_batched<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FL::bytes());
        if (e != cudaSuccess) return e;
      }
    }
    if constexpr (kFused) {
      cudaError_t e = cudaFuncSetAttribute(k_step_fused<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)FU::bytes());
      if (e != cudaSuccess) return e;
    }
    if constexpr (kLanes) {
      if constexpr (kBatched) {
        cudaError_t e = cudaFuncSetAttribute(k_volume_batched<EQ, N, R, 0>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_volume_batched<EQ, N, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PL::bytes());
        if (e != cudaSuccess) return e;
      }
      cudaError_t e = cudaFuncSetAttribute(k_volume_lanes_stage<EQ, N, R>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_volume_lanes<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    } else {
      cudaError_t e = cudaFuncSetAttribute(k_volume_tile_stage<EQ, N, R>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(k_volume_tile<EQ, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    }
  }
  static cudaError_t vol_batched(const BatchLaunch& b, cudaStream_t s) {
    if constexpr (kBatched) {
      if (b.shape == 1)
        k_volume_batched<EQ, N, R, 1><<<b.grid, LL::THREADS, PL::bytes(), s>>>(
            b.solves, b.tiles, b.ntiles, PPB<R>::get(b), PPB<R>::tab(b), b.slot);
      else
        k_volume_batched<EQ, N, R, 0><<<b.grid, LL::THREADS, PL::bytes(), s>>>(
            b.solves, b.tiles, b.ntiles, PPB<R>::get(b), PPB<R>::tab(b), b.slot);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static cudaError_t face_batched(const BatchLaunch& b, cudaStream_t s) {
    if constexpr (kBatched) {
      k_face_batched<EQ, N, R><<<b.grid, FL::THREADS, FL::bytes(), s>>>(b.solves, b.tiles, b.ntiles, PPB<R>::get(b),
                                                                        PPB<R>::tab(b), b.slot);
      return cudaGetLastError();
    }
    return cudaErrorNotSupported;
  }
  static int occupancy(int which, int shape) {
    int nb = 0;
    if constexpr (kBatched) {
      if (which == 0) {
        auto k = shape == 1 ? k_volume_batched<EQ, N, R, 1> : k_volume_batched<EQ, N, R, 0>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, LL::THREADS, PL::bytes());
      } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_face_batched<EQ, N, R>, FL::THREADS, FL::bytes());
      }
    }
    return nb;
  }
  static void fill(VariantOps* o) {
    o->vol_batched = kBatched ? &vol_batched : nullptr;
    o->face_batched = kBatched ? &face_batched : nullptr;
    o->occupancy = kBatched ? &occupancy : nullptr;
    o->vol_shapes = kBatched ? 2 : 0;
    o->threads_vol = LL::THREADS;
    o->threads_face = kFaceLanes ? FL::THREADS : 0;
    o->M = EQ::M;
    o->NP = L::NP;
    o->NF = L::NF;
    o->C = trace_comps<EQ>();
    o->ncs_per_elem = EQ::NCS ? ncs_values_per_elem<EQ, N>() : 0;
    o->dim = EQ::DIM;
    o->vol_bytes_per_elem = L::bytes_per_elem();
    o->lanes = kLanes;
    o->vol_smem = &vol_smem;
    o->real_bytes = sizeof(R);
    o->volume = &volume;
    o->face_update = &face_update;
    o->volume_stage = &volume_stage;
    o->face_stage = &face_stage;
    o->lambda = &lambda;
    o->step_fused = kFused ? &step_fused : nullptr;
    o->alpha = EQ::NC ? nullptr : &alpha;
    o->face_limited = EQ::NC ? nullptr : &face_limited;
    o->volume_ind = kVolInd ? &volume_ind : nullptr;
    o->alpha_smooth = EQ::NC ? nullptr : &alpha_smooth;
    o->totals = &totals;
    o->set_smem = &set_smem;
  }
};

template <class EQ, typename R>
bool fill_ops(int N, VariantOps* o) {
  switch (N) {
    case 1: Variant<EQ, 1, R>::fill(o); return true;
    case 2: Variant<EQ, 2, R>::fill(o); return true;
    case 3: Variant<EQ, 3, R>::fill(o); return true;
    case 4: Variant<EQ, 4, R>::fill(o); return true;
    case 5: Variant<EQ, 5, R>::fill(o); return true;
  }
  return false;
}

}  // namespace crk
