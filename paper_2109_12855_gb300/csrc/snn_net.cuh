// snn_net.cuh -- host-side definition of a net (shared by the C ABI and the
// serving loop).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "snn_internal.cuh"

using namespace snn;

namespace snn {
// Message returned by snn_last_error() on this thread.
void set_last_error(const char* msg);
// Tile geometry the store builder uses for n targets (see snn_api.cu).
void tile_geometry(uint32_t n, int window, int32_t hint, uint32_t* tile_w,
                   int* lo_bits, uint32_t* n_tiles);
// Device memory from the library's stream-ordered pool of the current
// device (see snn_api.cu); free with pool_free on a stream ordered after
// the last use.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
void pool_free(void* p, cudaStream_t s);
// Keep (+1) or let go (-1) of the device's pool: while held, memory freed by
// destroyed nets stays in the pool for the next ones (a server holds it for
// its lifetime, so that admitting a request never waits for memory to be
// mapped again).
void pool_hold(int dev, int delta);
// snn_simulate's asynchronous production path (serving uses it directly:
// may_capture false keeps it from instantiating a graph while builds run).
int simulate_async(snn_net* net, int64_t n_steps, bool may_capture);
}  // namespace snn

// The net: parameters, device buffers and host bookkeeping.
struct snn_net {
  snn_params p{};
  cudaStream_t stream = nullptr;
  bool counted = false;  // counted among the device's live nets
  bool own_stream = false;
  int device = 0;
  uint32_t n = 0, pitch = 0;
  uint32_t n_src = 0, g0 = 0;  // store rows (all sources); first neuron
  int fmt = 0, n_slots = 0;
  UpdConst uc{};
  float *V = nullptr, *I = nullptr, *J = nullptr;
  int32_t* refr = nullptr;
  float* rb = nullptr;
  uint32_t* counts = nullptr;
  Ctl* ctl = nullptr;
  uint64_t* row_ptr = nullptr;
  void* recs = nullptr;
  uint64_t n_syn = 0, recs_bytes = 0;
  uint32_t* tile_off = nullptr;  // [n][n_tiles + 1]
  bool check_noted = false;      // SNN_ERRF_CHECK counted (checked builds)
  uint32_t* xbuf = nullptr;      // caller's exchange buffer (snn_set_exchange)
  uint32_t xcap = 0;
  const void* x_parts_ok = nullptr;  // last gathered-parts pointer validated
  uint32_t tile_w = 0, n_tiles = 0;
  uint32_t pl_tiles = 0, tile_grp = 1;  // see NetView
  int lo_bits = 0;
  int window = 0;
  uint32_t mult_max = 0, k_in_max = 0, spikes_per_iv = 1;
  int acc_words = 2, acc_qs_min = 0;  // accumulator cells (see NetView)
  float max_abs_w = 0.f;
  SpikeEntry* list = nullptr;
  uint64_t list_cap = 0;
  SpikeEntry* ext_list = nullptr;
  uint32_t* ext_src = nullptr;
  int32_t* ext_t = nullptr;
  uint64_t ext_cap = 0;
  uint32_t* log_src = nullptr;
  int32_t* log_t = nullptr;
  uint64_t log_cap = 0;
  bool connected = false, finalized = false, pending = false;
  int interval = 0, dmin = 0, dmax = 0;
  long long t_host = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev;
  double ms_update = 0, ms_deliver = 0;
  uint64_t launches = 0, upd_launches = 0, del_launches = 0;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_prof = nullptr;  // the same intervals with timing events
  // STDP (snn_set_stdp): parameters and device state (StdpView)
  bool stdp_on = false;
  snn_stdp_params stdp{};
  StdpView sp{};
  // long-run spike statistics
  int32_t* isi_last = nullptr;
  uint32_t* isi_spikes = nullptr;
  uint32_t* isi_n = nullptr;
  double* isi_sum = nullptr;
  double* isi_sq = nullptr;

  NetView view() const {
    NetView v;
    v.n = n;
    v.n_src = n_src;
    v.g0 = g0;
    v.pitch = pitch;
    v.slot_mask = (uint32_t)n_slots - 1u;
    v.chunk = (uint32_t)chunk_records(fmt);
    v.fmt = fmt;
    v.V = V;
    v.I = I;
    v.J = J;
    v.refr = refr;
    v.rb = rb;
    v.counts = counts;
    v.row_ptr = row_ptr;
    v.recs = recs;
    v.tile_off = tile_off;
    v.tile_w = tile_w;
    v.n_tiles = n_tiles;
    v.pl_tiles = pl_tiles ? pl_tiles : n_tiles;
    v.tile_grp = tile_grp ? tile_grp : 1u;
    v.d_min = dmin;
    v.d_max = dmax;
    v.window = window;
    v.mult_max = mult_max;
    v.k_in_max = k_in_max;
    v.spikes_per_iv = spikes_per_iv;
    v.max_abs_w = max_abs_w;
    v.acc_words = acc_words;
    v.acc_qs_min = acc_qs_min;
    v.mean_run = n_src && n_tiles ? (float)((double)n_syn / ((double)n_src * n_tiles))
                                  : 0.f;
    v.list = list;
    v.list_cap = list_cap;
    v.xbuf = xbuf;
    v.xcap = xcap;
    v.gx = nullptr;
    v.gx_parts = 0;
    v.gx_stride = 0;
    v.gx_cap = 0;
    v.log_src = log_src;
    v.log_t = log_t;
    v.log_cap = log_cap;
    v.ctl = ctl;
    v.plastic = stdp_on && sp.wp != nullptr;
    v.sp = sp;
    v.isi_last = isi_last;
    v.isi_spikes = isi_spikes;
    v.isi_n = isi_n;
    v.isi_sum = isi_sum;
    v.isi_sq = isi_sq;
    return v;
  }
};

