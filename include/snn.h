/*
 * snn.h -- C ABI of libsnn: spike delivery and neuron update for a
 * time-driven simulation of a balanced random network of current-based
 * leaky integrate-and-fire neurons with alpha-shaped synaptic currents,
 * on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one studied in arXiv 2109.12855 ("Routing brain traffic
 * through the von Neumann bottleneck"): neurons are updated on a fixed time
 * grid (Section 2.1); once per min-delay interval the spikes emitted in that
 * interval are delivered, each spike walking its source's target segment
 * and adding every synapse's weight into the target neuron's spike ring
 * buffer at (emission step + delay) (Section 3.2, Algorithm REF; Section 3.1,
 * Fig. 3 for the data structures).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status: SNN_OK (0) or a negative SNN_E_* code.
 *    snn_last_error() returns a message for the calling thread's last error.
 *  - A net handle is opaque; the library owns all device memory behind it
 *    (allocated with cudaMalloc on the current device at snn_create and at
 *    connection time) and frees it in snn_destroy.
 *  - Caller buffers are borrowed for the duration of the call only.  Each
 *    buffer argument is accompanied by a `mem` flag: SNN_MEM_HOST (pageable
 *    or pinned host memory) or SNN_MEM_DEVICE (device memory of the net's
 *    device, e.g. a PyTorch CUDA tensor's data pointer).
 *  - Work is enqueued on the stream given to snn_create (a cudaStream_t
 *    passed as void*; NULL is the legacy default stream).  Calls that write
 *    to host memory, or return counts, synchronise that stream; all others
 *    are asynchronous.
 *  - Neuron i in [0, n_exc) is excitatory, [n_exc, n_exc + n_inh) inhibitory.
 *  - Time is counted in integer grid steps of h ms.  The ring buffer has
 *    n_slots slots (a power of two); absolute step u uses slot u mod n_slots.
 *  - Not thread-safe per net: one host thread at a time per handle.
 */
#ifndef SNN_H
#define SNN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNN_ABI_VERSION 1

/* Status codes. */
enum {
  SNN_OK = 0,
  SNN_E_OOM = -1,      /* device or host allocation failed */
  SNN_E_ARG = -2,      /* invalid argument (null pointer, size, range) */
  SNN_E_STATE = -3,    /* call not valid in the net's current state */
  SNN_E_TIMEOUT = -4,  /* a bounded device wait gave up */
  SNN_E_OVERFLOW = -5, /* an output did not fit; data was truncated */
  SNN_E_CUDA = -6      /* a CUDA runtime call failed */
};

/* Memory kinds for caller buffers. */
enum { SNN_MEM_HOST = 0, SNN_MEM_DEVICE = 1 };

/* Synapse record formats of the connection store.
 *  SNN_W_FP32_12B: 12 bytes {uint32 target; float32 weight; uint8 delay;
 *                  3 pad bytes}.
 *  SNN_W_BF16_8B:  8 bytes {uint32 target; uint8 delay; uint8 pad;
 *                  bfloat16 weight}; weights are rounded FP64 -> BF16 to
 *                  nearest, ties to even, in one step.
 * Both accumulate into a float32 ring buffer. */
enum { SNN_W_FP32_12B = 0, SNN_W_BF16_8B = 1 };

/* Delivery kernels.
 *  SNN_DELIVER_TILED: targets are cut into tiles of about N / (k * #SMs)
 *    neurons (k the smallest integer for which a tile's ring-buffer window
 *    fits in shared memory); each segment is stored sorted by (tile, delay,
 *    target) with a per-row tile index, and one CTA per tile accumulates
 *    the interval's events for its targets in shared memory, then adds them
 *    into the ring buffer without global atomics.
 *  SNN_DELIVER_ATOMIC: every event is one red.global.add.f32 (merge-path
 *    split of the interval's chunks over all warps). */
enum { SNN_DELIVER_TILED = 0, SNN_DELIVER_ATOMIC = 1 };

/* Device error flags (snn_stats.error_flags, sticky until snn_clear_errors). */
enum {
  SNN_ERRF_SPIKE_LIST = 1u << 0, /* interval spike list overflowed */
  SNN_ERRF_SPIKE_LOG = 1u << 1,  /* spike recording log overflowed */
  SNN_ERRF_BAD_SOURCE = 1u << 2, /* external spike with source >= N */
  SNN_ERRF_CHUNKS = 1u << 3,     /* chunk counter of one interval overflowed */
  SNN_ERRF_TIMEOUT = 1u << 4,    /* a bounded device wait gave up (delivery of
                                    that launch is incomplete) */
  SNN_ERRF_SCALES = 1u << 5,     /* internal: an interval's exact-sum scales
                                    were proven on the host but not found on
                                    the device (never expected) */
  SNN_ERRF_CHECK = 1u << 6       /* bounds-checked builds only (snn_checked):
                                    a synapse record with a target or delay
                                    outside the store's ranges, a tile index
                                    entry outside its row, or a spike list
                                    with decreasing chunk offsets was skipped */
};

/* Neuron model and simulation parameters (iaf_psc_alpha, resting potential
 * 0 mV; Section 1 and Section 2.1 of the paper: linear subthreshold
 * dynamics integrated exactly, threshold, reset, refractory period).
 *   dV/dt = -V/tau_m + I/C;  dI/dt = -I/tau_syn + J;  dJ/dt = -J/tau_syn;
 *   an arriving weight w (pA) adds (e/tau_syn) w to J (PSC peak = w).
 * One step t: (1) V <- P31 J + P32 I + P33 V unless refractory (then the
 * refractory count decreases); (2) I <- P21 J + P22 I, J <- P11 J;
 * (3) J += (e/tau_syn)(rb[t] + w_ext * Poisson(nu_ext h)), rb[t] <- 0;
 * (4) if V >= v_th: V <- v_reset, refractory for round(t_ref/h) steps, spike.
 * State is float32 on the device; the propagator entries are computed in
 * FP64 on the host once and rounded to float32. */
typedef struct snn_params {
  uint32_t n_exc, n_inh;  /* population sizes; n_exc + n_inh in [1, 2^24) */
  double h;               /* grid step, ms (> 0) */
  double tau_m;           /* membrane time constant, ms */
  double c_m;             /* membrane capacitance, pF */
  double v_th;            /* threshold, mV */
  double v_reset;         /* reset potential, mV */
  double t_ref;           /* refractory period, ms */
  double tau_syn;         /* synaptic time constant, ms (!= tau_m) */
  double nu_ext;          /* Poisson drive rate per neuron, Hz (>= 0) */
  double w_ext;           /* weight of one drive spike, pA */
  uint64_t seed;          /* initial potentials (stream 1), drive (stream 2) */
  int32_t weight_format;  /* SNN_W_FP32_12B or SNN_W_BF16_8B */
  int32_t n_slots;        /* ring-buffer slots: power of two in [2, 256] */
  int32_t interval;       /* steps per update/deliver interval; 0 = the
                             minimum delay of the connections */
  int32_t init_v_random;  /* 1: V0 ~ U[v_reset, v_th) from Philox stream 1;
                             0: V0 = 0 */
  int32_t count_events;   /* 1: keep a uint32 [n_slots][N] per-cell count of
                             delivered events (test instrument) */
  int32_t deliver_mode;   /* SNN_DELIVER_TILED (0, default) or
                             SNN_DELIVER_ATOMIC (1); see below */
  uint64_t spike_log_capacity; /* entries kept for snn_read_spikes (0: none) */
  int32_t tile_width;     /* targets per tile of the tiled delivery; 0 = the
                             automatic choice (about N / #SMs), otherwise used
                             as given when its shared-memory window fits */
  int32_t stream_priority; /* priority of the stream the library creates for
                             the net when none is given (0: default; see
                             cudaDeviceGetStreamPriorityRange: larger is
                             lower priority) */
  uint32_t part_lo, part_hi; /* target partition: this net holds neurons
                             [part_lo, part_hi) of the population of n_exc +
                             n_inh neurons and the synapses of all sources
                             onto them (0, 0: the whole population).  Neuron
                             indices in spike lists, the spike log and the
                             random streams are global; state and ring-buffer
                             arrays are local (part_hi - part_lo entries).
                             Partitions exchange their interval lists (see
                             snn_read_pending) and agree on the accumulation
                             bounds (snn_get_bounds / snn_set_bounds) so that
                             their union equals the whole net bit for bit. */
  int32_t acc_words;      /* words per cell of the tiled delivery's exact
                             accumulator: 0 = automatic (one word for a BF16
                             store when the connection rule proves that every
                             stored weight is a multiple of the smallest
                             fixed-point step an interval's spike list can
                             need, which halves the shared memory per target;
                             else two), 2 = always two.  Both give the same
                             sums. */
  int32_t build_yield;    /* 1: the connection-store build runs as short
                             CTAs that each fill a whole SM, so that an SM
                             is entirely free whenever one ends and kernels
                             of higher-priority streams (nets already
                             running, whose delivery CTAs need a whole SM)
                             get it first; the build itself is somewhat
                             slower.  0: the normal shape.  The server sets 1
                             for the nets it builds beside running ones. */
} snn_params;

/* Fixed in-degree connection rule (the benchmark model's random
 * connectivity, Section 2.2).  Every target j draws k_exc sources uniformly
 * from the excitatory and k_inh from the inhibitory population, with
 * replacement (multapses and autapses allowed).  Draw k of target j uses
 * Philox4x32-10 (Salmon et al., SC'11) with counter (j, k, 0, 0) and key
 * (seed low, seed high): word 0 -> source floor(u N_pop 2^-32) (+ n_exc for
 * inhibitory draws, k >= k_exc), word 1 -> delay d_lo + floor(u (d_hi-d_lo+1)
 * 2^-32) steps, words 2, 3 -> Box-Muller normal z when sd != 0 (w = mean +
 * sd z, computed in FP64, then clipped if requested, then rounded to the
 * store's format). */
typedef struct snn_conn_params {
  uint32_t k_exc, k_inh;  /* in-degree per target from each population */
  double w_exc, w_inh;    /* mean weights, pA */
  double sd_exc, sd_inh;  /* weight standard deviations, pA (0: fixed) */
  int32_t d_lo, d_hi;     /* delay range in steps, 1 <= d_lo <= d_hi <= n_slots,
                             d_hi <= 255 */
  uint64_t seed;          /* connectivity key */
  int32_t clip_exc;       /* 1: excitatory weights clipped at >= 0 */
  int32_t clip_inh;       /* 1: inhibitory weights clipped at <= 0 */
} snn_conn_params;

/* Counters and timings of a net. */
typedef struct snn_stats {
  uint64_t events_delivered; /* synaptic events added into ring buffers */
  uint64_t spikes;           /* spikes emitted by snn_update/snn_simulate */
  uint64_t n_synapses;       /* synapses in the store */
  int64_t t_now;             /* next step to be updated */
  int32_t interval;          /* steps per interval */
  int32_t min_delay, max_delay;
  uint32_t error_flags;      /* SNN_ERRF_* */
  uint64_t kernel_launches;  /* library kernels launched since creation */
  uint64_t update_launches, deliver_launches;
  double ms_update, ms_deliver; /* CUDA-event times while profiling is on */
  uint64_t bytes_per_record;    /* 12 or 8 */
  uint64_t store_bytes;         /* device bytes of the record array */
  uint32_t n_tiles, tile_width; /* target tiles of the store */
  int32_t window;               /* ring steps one interval reaches */
  int32_t deliver_mode;         /* kernel used by update/simulate */
  uint64_t plastic_events;      /* plastic weight updates (STDP nets) */
  uint64_t stdp_truncated;      /* of which the post-spike window reached
                                   past the kept history (see snn_set_stdp) */
  uint32_t first_neuron;        /* global index of local neuron 0 */
  uint32_t n_sources;           /* rows of the store (the whole population) */
  int32_t acc_words;            /* words per accumulator cell (1 or 2) */
  int32_t reserved_;
} snn_stats;

/* Bounds of one delivery launch's exact accumulation (see snn_set_bounds). */
typedef struct snn_bounds {
  uint32_t mult_max;  /* most synapses sharing (source, target, delay) */
  uint32_t k_in_max;  /* largest in-degree */
  float max_abs_w;    /* largest |weight| */
  uint32_t reserved_; /* 0 */
} snn_bounds;

/* Pair-based power-law STDP of the excitatory-to-excitatory synapses
 * (arXiv 2109.12855, Section 6: plasticity as an update scheme driven by
 * presynaptic spikes, weights computed when a spike becomes visible at the
 * target; the cited Morrison et al. 2007 rule).  A synapse i->j with delay d
 * sees a pre spike at its emission step t_e and a post spike of j at t_p + d;
 * every pair interacts with D = (t_p + d - t_e) h: D > 0 potentiates by
 * lambda w0^(1-mu) w^mu exp(-D/tau_plus), D <= 0 depresses by
 * lambda alpha w exp(D/tau_minus).  At each delivered pre spike the weight
 * first takes, in time order, the potentiation owed to the post spikes seen
 * since the previous pre spike, then the depression, and is kept in
 * [0, w_max]; the delivered value is the new weight. */
typedef struct snn_stdp_params {
  double tau_plus, tau_minus;  /* ms */
  double lambda, alpha, mu;
  double w0;                   /* pA: weight scale of the power law */
  double w_max;                /* pA: upper bound (also bounds the exact
                                  accumulation of the delivery kernel) */
  int32_t history;             /* post spikes kept per neuron: a power of
                                  two, 2..32; a
                                  window that reaches past them is counted
                                  in snn_stats.stdp_truncated */
  int32_t reserved_;           /* 0 */
} snn_stdp_params;

typedef struct snn_net snn_net;

/* Library identity and diagnostics. */
int snn_abi_version(void);
const char* snn_last_error(void);
/* Host-side fault injection for tests (not part of the paper's method):
 * after `after` more device allocations of the library succeed (process-
 * wide, any thread), the next `count` fail as if device memory were
 * exhausted, so that error paths (SNN_E_OOM from snn_create, connect,
 * finalize, a server's build) run without exhausting the GPU.  after < 0
 * switches it off. */
int snn_debug_fail_allocations(int64_t after, int64_t count);

/* Fill *p with the benchmark defaults: 1,000 E + 250 I neurons, h = 0.1 ms,
 * tau_m = 10 ms, C = 250 pF, V_th = 20 mV, V_reset = 0, t_ref = 2 ms,
 * tau_syn = 0.5 ms, no drive, FP32 records, 32 slots, random V0. */
int snn_default_params(snn_params* p);

/* PSC amplitude w (pA) whose membrane response peaks at psp_mv (mV) for the
 * neuron model in *p ("J = 0.1 mV" weights of the benchmark model are given
 * as peak PSP amplitudes).  Host-only arithmetic; needs no GPU. */
int snn_psc_weight_for_psp(const snn_params* p, double psp_mv, double* w_pa);

/* Create a net on the current CUDA device.  Allocates neuron state (SoA
 * float32 V, I, J and int32 refractory counts), the ring buffer
 * rb[n_slots][N] (float32, zeroed) and, if requested, the event counts and
 * the spike log.  Initial V per init_v_random.  stream: cudaStream_t as
 * void*.  Errors: SNN_E_ARG (bad parameter), SNN_E_OOM, SNN_E_CUDA. */
int snn_create(const snn_params* p, void* stream, snn_net** out);

/* Build the connection store from the fixed in-degree rule (see
 * snn_conn_params) on the device: count out-degrees, prefix-sum them into
 * row offsets, scatter, sort every target segment by (delay, target, k) and
 * pack records (Section 3.1: source-specific target segments).  One connect
 * call per net.  Errors: SNN_E_STATE (already connected), SNN_E_ARG,
 * SNN_E_OOM. */
int snn_connect_fixed_indegree(snn_net* net, const snn_conn_params* c);

/* Build the store from an explicit edge list of n edges: edge e connects
 * src[e] -> tgt[e] with delay[e] steps (1 <= delay <= min(n_slots, 255)) and
 * weight w[e] pA (rounded to the store's format).  Segments are sorted by
 * (delay, target, e).  Requires n < 2^32.  mem: where the four arrays live.
 * Errors: SNN_E_STATE, SNN_E_ARG (index or delay out of range), SNN_E_OOM. */
int snn_connect_edges(snn_net* net, const uint32_t* src, const uint32_t* tgt,
                      const uint8_t* delay, const double* w, uint64_t n,
                      int mem);

/* Freeze the store and size the interval buffers: interval = params.interval
 * or the minimum delay (n_slots when there are no synapses); requires
 * interval <= min delay and max delay <= n_slots.  Must precede update,
 * deliver and simulate.  Errors: SNN_E_STATE, SNN_E_ARG, SNN_E_OOM. */
int snn_finalize(snn_net* net);

/* Update all neurons for n_steps (1 <= n_steps <= interval) grid steps
 * starting at absolute step t0 (Section 2.1), reading and clearing ring
 * buffer slots t0 .. t0+n_steps-1.  Spikes go to the pending interval list
 * (and to the log).  t0 = SNN_T_DEVICE starts at the net's device clock
 * (where the last delivery left it) instead: the call then reads no host
 * time, so an update + exchange + delivery sequence can be captured into a
 * CUDA graph and replayed (the library's host copy of the clock is not
 * advanced by replays).  Errors: SNN_E_STATE if spikes of an earlier update
 * are still pending (deliver or discard them first), SNN_E_ARG. */
#define SNN_T_DEVICE (-1)
int snn_update(snn_net* net, int64_t t0, int32_t n_steps);

/* Deliver the pending interval list produced by snn_update (Algorithm REF
 * semantics), or drop it.  Asynchronous. */
int snn_deliver_pending(snn_net* net);
int snn_discard_pending(snn_net* net);

/* Deliver an external spike list (Section 3.2, Algorithm REF): for every
 * spike s and every synapse (src[s] -> target, delay d, weight w) in the
 * source's segment, rb[(t_emit[s] + d) mod n_slots][target] += w in float32.
 * src, t_emit: n_spikes entries in `mem` memory; duplicates allowed.
 * n_events_out (optional, host): number of additions; when non-null the
 * call synchronises.  A source >= N is skipped and sets SNN_ERRF_BAD_SOURCE
 * (host inputs are checked up front and give SNN_E_ARG). */
int snn_deliver(snn_net* net, const uint32_t* src, const int32_t* t_emit,
                uint32_t n_spikes, int mem, uint64_t* n_events_out);

/* Same delivery as snn_deliver, for callers that cannot let the library
 * allocate device memory: processes whose device memory is fully reserved
 * by another allocator, or latency-critical loops where cudaMalloc's implicit
 * device synchronisation is not acceptable.  (The paper has no counterpart:
 * this is a deployment variant of the delivery entry point.)
 *
 * The caller's list is staged in a fixed scratch array that every GPU
 * loading the library holds until the process exits (SNN_NOALLOC_MAX_SPIKES
 * entries of 16 bytes = 4 MiB); the call itself allocates nothing.
 *  - src, t_emit: n_spikes entries in DEVICE memory (no host staging).
 *  - n_spikes > SNN_NOALLOC_MAX_SPIKES is rejected with SNN_E_ARG.
 *  - The first call on a device looks up the scratch's device address; make
 *    that first call before any stream capture.  The address is kept for
 *    the life of the process: after cudaDeviceReset on that device the entry
 *    point must not be called again in the same process.
 *  - src and t_emit must be device (or managed) memory of the net's device;
 *    anything else is refused with SNN_E_ARG before any work is queued.
 *  - All calls share the scratch: calls whose GPU work overlaps (different
 *    streams, or other host threads) race and must be serialised by the
 *    caller.  Counters that must start at zero are cleared by every call.
 *  - n_events_out (optional, host): additions made; when non-null the call
 *    synchronises the net's stream.
 * Errors: SNN_E_ARG, SNN_E_STATE (not finalized), SNN_E_CUDA. */
#define SNN_NOALLOC_MAX_SPIKES (1u << 18)
int snn_deliver_noalloc(snn_net* net, const uint32_t* src,
                        const int32_t* t_emit, uint32_t n_spikes,
                        uint64_t* n_events_out);

/* Advance the net by n_steps grid steps from its current time: repeat
 * {update one interval; deliver its spikes} (the time-driven cycle of
 * Section 1); the last interval may be shorter.  Full intervals run as
 * captured CUDA graphs unless profiling is on.  Asynchronous. */
int snn_simulate(snn_net* net, int64_t n_steps);

/* Copy up to cap logged spikes (source, step) in emission-interval order
 * (order within an interval unspecified) into src/t and clear the log;
 * *n receives the number logged (> cap: the rest are dropped and the call
 * returns SNN_E_OVERFLOW).  Synchronises. */
int snn_read_spikes(snn_net* net, uint32_t* src, int32_t* t, uint64_t cap,
                    uint64_t* n, int mem);

/* Ring buffer as float32 [n_slots][N] (row u holds slot u).  Read
 * synchronises for host memory. */
int snn_read_rb(snn_net* net, float* dst, int mem);
int snn_write_rb(snn_net* net, const float* src, int mem);
/* Event counts as uint32 [n_slots][N] (requires count_events). */
int snn_read_counts(snn_net* net, uint32_t* dst, int mem);
/* Zero the ring buffer and the event counts. */
int snn_clear_rb(snn_net* net);

/* Neuron state, N entries each (float32 V mV, I pA, J pA/ms; int32
 * remaining refractory steps).  Any pointer may be NULL to skip it. */
int snn_read_state(snn_net* net, float* V, float* I, float* J, int32_t* refr,
                   int mem);
int snn_write_state(snn_net* net, const float* V, const float* I,
                    const float* J, const int32_t* refr, int mem);

/* Enable STDP (see snn_stdp_params) on the E->E synapses; call after
 * snn_create and before connecting.  Plastic nets need the tiled delivery
 * (deliver_mode SNN_DELIVER_TILED) and at most one spike per neuron per
 * interval (round(t_ref/h) + 1 >= interval, checked at snn_finalize).  The
 * traces are kept by snn_update, so caller spike lists (snn_deliver,
 * snn_deliver_noalloc) and checkpoints are refused with SNN_E_STATE.
 * Weights start at the stored weights and change as plastic deliveries run;
 * read them with snn_read_weights.  SNN_E_ARG for bad parameters,
 * SNN_E_STATE if the net is already connected. */
int snn_set_stdp(snn_net* net, const snn_stdp_params* p);

/* The pending interval list of the last snn_update (before its delivery):
 * global source indices and emission steps, n entries (*n; up to cap are
 * copied).  Partitions gather these lists from each other (all-gather) and
 * deliver the union to themselves with snn_deliver after
 * snn_discard_pending.  mem: SNN_MEM_HOST or SNN_MEM_DEVICE for src / t.
 * Synchronises.  SNN_E_STATE without a pending update, SNN_E_OVERFLOW when
 * n > cap. */
int snn_read_pending(snn_net* net, uint32_t* src, int32_t* t, uint64_t cap,
                     uint64_t* n, int32_t mem);

/* Deliver the spike list gathered from all partitions of a partitioned
 * network as this interval's list: like snn_deliver_pending, with the
 * pending list of the last snn_update replaced by src / t (global sources;
 * host or device memory per mem).  The list must be an interval list (every
 * neuron at most once per refractory period plus one step), so the same
 * accumulation bounds as snn_deliver_pending apply and a partition sums
 * exactly as the whole net does.  Advances the clock; *n_events_out (may be
 * NULL) receives the events delivered into this partition.  SNN_E_STATE
 * without a pending update, SNN_E_OVERFLOW beyond N x interval spikes. */
int snn_deliver_gathered(snn_net* net, const uint32_t* src,
                         const int32_t* t_emit, uint32_t n_spikes, int mem,
                         uint64_t* n_events_out);

/* Device-resident spike exchange between partitions (Section 2.1: the
 * spikes of one min-delay interval are exchanged between processes once,
 * before their delivery).  Without any host round trip per interval:
 *
 *   snn_update(part, t0, n)          writes the interval's own spikes into
 *                                    the part's exchange buffer too
 *   all-gather of the fixed-size     (NCCL on the caller's stream, or a
 *   exchange buffers of all parts     plain device copy within one process)
 *   snn_deliver_exchanged(part, ...) delivers the union read directly from
 *                                    the gathered buffers
 *
 * Exchange buffer layout (little-endian 32-bit words, 16-byte aligned
 * device memory of the net's device, 16 + 8 cap bytes):
 *   word 0          spike count of the interval: the update adds its
 *                   spikes, the interval's delivery (snn_deliver_pending,
 *                   snn_simulate, snn_deliver_gathered or
 *                   snn_deliver_exchanged) clears it when it completes;
 *                   snn_set_exchange and snn_discard_pending zero it
 *   words 1..3      unused (alignment)
 *   words 4 + 2k    entry k: global source index
 *   words 5 + 2k    entry k: emission step (int32)
 * A count above cap (an undersized buffer) keeps the first cap entries and
 * raises SNN_ERRF_SPIKE_LIST; snn_exchange_capacity gives the capacity that
 * can never overflow.  Since a net's delivery clears its own buffer, other
 * nets read it only through a copy taken before that delivery (the
 * all-gather's output; in one process, a device copy), while a net may read
 * its own attached buffer in place. */

/* Entries an exchange buffer of this partition needs so that it never
 * overflows: local neurons x most spikes a neuron emits per interval (one
 * per refractory period plus one step).  Finalized nets. */
int snn_exchange_capacity(snn_net* net, uint64_t* cap_entries);

/* Attach (buf != NULL) or detach (buf == NULL) the caller-owned exchange
 * buffer of cap_entries entries (layout above; buf 16-byte aligned device
 * memory of the net's device; not freed by the library).  While attached
 * every snn_update / snn_simulate interval also writes its spikes there.
 * SNN_E_ARG for a host, misaligned or foreign pointer or cap_entries of 0
 * or above 2^32 - 1; SNN_E_STATE before snn_finalize or with an update
 * pending. */
int snn_set_exchange(snn_net* net, void* buf, uint64_t cap_entries);

/* Deliver the pending interval with the list gathered from n_parts
 * exchange buffers, part p at parts + p x stride_bytes (device memory; each
 * holds its own count, so parts may be filled to different lengths; a count
 * above (stride_bytes - 16) / 8 is read as that many entries).  The union is
 * delivered as snn_deliver_gathered would deliver it (identical ring
 * buffers).  The events delivered into this partition are
 * counted on the device (snn_get_stats).  Asynchronous on the net's stream:
 * the gathered buffers must be complete in stream order (e.g. an NCCL
 * all-gather on the same stream) and stay unchanged until the delivery
 * finishes.  Needs the tiled delivery and a static (non-plastic) net.
 * SNN_E_STATE without a pending update, in atomic delivery mode or for
 * plastic nets; SNN_E_ARG for n_parts outside [1, 64], a misaligned parts
 * pointer or stride, or a stride below 16 bytes. */
int snn_deliver_exchanged(snn_net* net, const void* parts, uint32_t n_parts,
                          uint64_t stride_bytes);

/* Accumulation bounds of the store (finalized nets).  The tiled delivery
 * sums each ring-buffer cell exactly in fixed point with scales derived
 * from these bounds; partitions of one network take the maximum of their
 * bounds (snn_set_bounds raises each field to at least the given value) so
 * that they round every event the way the whole net does. */
int snn_get_bounds(snn_net* net, snn_bounds* out);
int snn_set_bounds(snn_net* net, const snn_bounds* b);

/* Long-run spike statistics, kept per neuron by snn_update / snn_simulate
 * (not by the batched steps of a server): spikes counted, inter-spike
 * intervals counted, and FP64 sums of the intervals and of their squares,
 * in steps (integers, so the sums are exact below 2^53).  The mean rate is
 * n_spikes / time and the CV of the intervals sqrt(sq/n - (sum/n)^2) /
 * (sum/n).  Host arrays of N entries (any may be NULL); synchronises. */
int snn_read_spike_stats(snn_net* net, uint32_t* n_spikes, uint32_t* n_isi,
                         double* isi_sum, double* isi_sq);
/* Zero the counts and sums (the latest spike times are kept, so the first
 * interval after a clear is counted whole). */
int snn_clear_spike_stats(snn_net* net);

/* Current weight of every synapse in store order (the order of
 * snn_read_store): n_synapses floats into w (host or device memory per
 * mem).  Static synapses return their stored weight. */
int snn_read_weights(snn_net* net, float* w, int32_t mem);

/* The finalized store: row_ptr uint64 [N+1]; per synapse target uint32,
 * delay uint8 and weight widened to float32 (n_synapses entries each).
 * Synchronises for host memory. */
int snn_read_store(snn_net* net, uint64_t* row_ptr, uint32_t* tgt,
                   uint8_t* delay, float* w, int mem);

/* Replace the Poisson drive (rate nu_ext Hz, weight w_ext pA per drive
 * spike) from the next update on.  Errors: SNN_E_ARG (negative rate, or a
 * rate whose inversion table exceeds 128 outcomes). */
int snn_set_drive(snn_net* net, double nu_ext, double w_ext);
/* Checkpoint / restore of the dynamic state: V, I, J, refractory counts,
 * the ring buffer and the clock.  Every random draw is a Philox call keyed by
 * (neuron, step) and the seed, so no generator state exists beyond the
 * clock.  The connection store and parameters are not included: restore into
 * a net built with the same parameters and connections.  The image is a
 * little-endian byte string: 64-byte header (magic "SNNSTATE", version, N,
 * n_slots, t_now), then float32 V, I, J, int32 refr (N each) and float32
 * rb[n_slots][N].  snn_state_size gives its length; save synchronises;
 * load requires no pending spikes and checks the header (SNN_E_ARG on a
 * mismatch). */
int snn_state_size(snn_net* net, uint64_t* bytes);
int snn_save_state(snn_net* net, void* host_buf, uint64_t cap);
int snn_load_state(snn_net* net, const void* host_buf, uint64_t size);
/* Set the step counter (next step to update). */
int snn_set_time(snn_net* net, int64_t t);
/* Profiling on: every update and deliver launch is bracketed by CUDA events
 * on the net's stream; times accumulate into snn_stats.ms_update /
 * ms_deliver.  snn_simulate keeps its CUDA graphs of whole intervals, with
 * the events captured as graph nodes, so the kernels are timed in the launch
 * context of the production path (the host waits after each graph to read
 * the times); other calls record the events around plain launches. */
int snn_set_profiling(snn_net* net, int on);
/* Counters (synchronises). */
int snn_get_stats(snn_net* net, snn_stats* out);
int snn_clear_errors(snn_net* net);
/* Wait for all work of the net. */
int snn_sync(snn_net* net);
/* 1 for a bounds-checked build of the library (compiled with SNN_CHECK:
 * every record's target and delay, every tile index entry and the order of
 * every chunk offset is checked before use, failures raise SNN_ERRF_CHECK
 * and skip the access), 0 for the production build. */
int snn_checked(void);
/* Bounds-checked builds: the number of nets whose SNN_ERRF_CHECK flag was
 * seen set by snn_get_stats or snn_destroy since the library was loaded
 * (always 0 in production builds). */
uint64_t snn_debug_check_failures(void);
/* Bounds-checked builds only: overwrite the target (field 0) or delay
 * (field 1) of synapse record `index` of a finalized net with `value`, so
 * that tests can show the checks skip and flag a corrupt store.
 * SNN_E_STATE in production builds (whose kernels trust the store),
 * SNN_E_ARG for an index outside the store or an unknown field. */
int snn_debug_poke_record(snn_net* net, uint64_t index, int field,
                          uint32_t value);
/* Throughput probe of the L2 reductions that carry the ring-buffer
 * additions of Algorithm REF (Section 3.2: rb[(t + d) mod S][target] += w;
 * on the GPU one red.global.add.f32 per event in the atomic delivery, one
 * per nonzero window cell in the tiled delivery's flush).  Adds 1.0f
 * n_ops times into buf[n_cells]:
 *  - buf: n_cells floats of DEVICE memory owned by the caller (not
 *    cleared: each cell grows by the number of operations that hit it);
 *  - pattern SNN_PROBE_SCATTER: operation k hits a hash of k scaled to
 *    [0, n_cells) (scattered targets); SNN_PROBE_SWEEP: cell k mod n_cells
 *    (32 consecutive cells per warp, like the flush);
 *  - stream: a cudaStream_t (NULL: the legacy default stream); the call
 *    synchronises it and returns in *ms the CUDA-event time of the launch.
 * Errors: SNN_E_ARG (null or non-device buf, n_cells outside [1, 2^32),
 * n_ops 0, unknown pattern), SNN_E_CUDA. */
#define SNN_PROBE_SCATTER 0
#define SNN_PROBE_SWEEP 1
int snn_probe_reductions(float* buf, uint64_t n_cells, uint64_t n_ops,
                         int pattern, void* stream, float* ms);
/* The stream the net's work is enqueued on (*stream: a cudaStream_t; the
 * one given to snn_create, or the one the library created when none was
 * given).  Partitions that read each other's exchange buffers must share
 * one stream, or order theirs with events. */
int snn_get_stream(snn_net* net, void** stream);
/* Free everything; net may be NULL. */
int snn_destroy(snn_net* net);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent simulation requests.
 * (The paper has no serving layer; this is the deployment form of the same
 * update/deliver cycle.)
 *
 * A server owns a device-memory budget.  Submitted requests queue in
 * arrival order in one of two size classes (below 2^24 synapses, and the
 * rest); each class has a builder thread that admits its oldest request
 * once the estimated footprint fits the budget, and builds the connection
 * store on the net's own stream at the lowest stream priority while the
 * admitted nets keep running, so a small request never waits behind the
 * build of a large one.  Running nets are grouped into three lanes by
 * synapse count (< 2^24, < 2^27, the rest); each lane has its own stream
 * (smaller nets: higher priority), block -> net lookup tables and a wall-time
 * autotuner that picks how many intervals one step runs (1, 2, 4, 8 or 16).
 * Each snn_server_step advances every lane's nets by that many intervals in
 * ONE batched update launch and ONE batched tiled-delivery launch per
 * interval for all nets of the lane (per-net clock, state, store and
 * interval), replayed from a graph cached per interval count while the lane
 * is unchanged.  Nets that reached their step count are retired: their
 * counters (and spikes, if recorded) move to the request's result and their
 * memory is released.
 * Results do not depend on the mix: delivery sums are exact fixed point and
 * every random draw is keyed by (neuron, step), so a request's spikes are
 * bit-identical alone and batched.
 * Threads: submit, poll, spikes, release and get_stats may be called from
 * any thread; snn_server_step and snn_server_destroy from one thread at a
 * time (the serving loop).
 * ---------------------------------------------------------------------- */
typedef struct snn_server snn_server;

typedef struct snn_request {
  snn_params params;      /* model and seed; weight_format must equal the
                             server's; spike_log_capacity is set by the
                             server when record_spikes is 1 */
  snn_conn_params conn;   /* fixed in-degree connectivity (k_exc + k_inh >= 1) */
  int64_t n_steps;        /* biological time to simulate, in steps (>= 1) */
  uint64_t user_tag;      /* returned in the result */
  int32_t record_spikes;  /* 1: keep the spike list (snn_server_spikes) */
  int32_t pad_;
} snn_request;

enum {
  SNN_REQ_QUEUED = 0,
  SNN_REQ_BUILDING = 1,
  SNN_REQ_RUNNING = 2,
  SNN_REQ_DONE = 3,
  SNN_REQ_FAILED = -1,
  SNN_REQ_CANCELLED = 4
};

typedef struct snn_result {
  uint64_t id, user_tag;
  int32_t state;          /* SNN_REQ_* */
  int32_t error;          /* status code of a failed request */
  uint64_t n_neurons, n_synapses;
  uint64_t spikes, events; /* counters of the finished simulation */
  int64_t n_steps;
  double t_submit, t_admit, t_start, t_done; /* seconds on the server clock:
                             submitted, admitted (build begins), first batch
                             step, result ready */
  uint64_t bytes;         /* device bytes reserved for it */
} snn_result;

typedef struct snn_server_stats {
  uint64_t submitted, done, failed, active, queued;
  uint64_t steps, intervals, kernel_launches;
  uint64_t events, spikes;  /* of finished requests */
  uint64_t mem_budget, mem_used;
  int32_t intervals_per_step; /* autotuner's choice for the lane that
                                 ran the most intervals */
  int32_t tuned;              /* 1 once every lane that stepped settled */
  double gpu_ms;              /* CUDA-event time of the batched launches */
} snn_server_stats;

/* Create a server with a device-memory budget (bytes), one weight format
 * for all its requests, on the current device; stream: cudaStream_t as
 * void* for the batched launches (NULL: an internal blocking stream). */
int snn_server_create(uint64_t mem_budget, int32_t weight_format,
                      void* stream, snn_server** out);
/* Serving options (snn_server_set_option):
 *  SNN_SERVE_OPT_PERSISTENT  1: each snn_server_step is ONE launch
 *    of a persistent kernel that advances every running net by its own
 *    number of intervals: CTAs claim ready items -- a net's update blocks of
 *    an interval, then its delivery tiles -- from per-net device queues, an
 *    update once the net's previous delivery is complete, a delivery once
 *    its update is; nets are served smallest first, each net runs as many
 *    intervals as fit the step's target GPU time at its measured time per
 *    interval, and the target is autotuned (0.25 - 2 ms).  While a large
 *    request is being built, 16 SMs are left to the build.  0 (default): the
 *    lanes of batched update and delivery launches described above, which
 *    measure faster.  Changes only while no net runs (SNN_E_STATE
 *    otherwise).
 *  SNN_SERVE_OPT_SPIN_LIMIT  polls (32 to 256 ns apart) a CTA of the
 *    persistent kernel makes while no item is ready before it gives up:
 *    the launch then ends, the nets it ran fail with SNN_E_TIMEOUT
 *    (default 2^20, a fraction of a second).
 *  SNN_SERVE_OPT_STEP_US     target GPU time of a persistent step in
 *    microseconds (0: autotuned).
 *  SNN_SERVE_OPT_EXCLUSIVE   1: each step runs ONE net alone, with the
 *    single-net kernels and tiles (about one per SM) on the net's own
 *    stream, for about 1 ms of GPU time: the running net with the least
 *    remaining work (steps left x synapses; shortest remaining processing
 *    time first), chosen again at every step, so a newly admitted smaller
 *    request preempts a larger one within a step or two; two steps are kept
 *    queued so that the GPU does not idle between them.  Builds still run
 *    concurrently.  0 (default): lanes.  Changes only while no net runs
 *    (SNN_E_STATE otherwise). */
enum {
  SNN_SERVE_OPT_PERSISTENT = 0,
  SNN_SERVE_OPT_SPIN_LIMIT = 1,
  SNN_SERVE_OPT_STEP_US = 2,
  SNN_SERVE_OPT_EXCLUSIVE = 3
};
int snn_server_set_option(snn_server* sv, int32_t option, double value);

/* Queue a request; *id identifies it.  Thread-safe.  SNN_E_ARG for invalid
 * parameters or a footprint above the whole budget.  A request with
 * params.tile_width == 0 gets delivery tiles in proportion to its synapses
 * (about one per 4.2e6, at most one per SM), since all served nets share
 * each delivery launch. */
int snn_server_submit(snn_server* sv, const snn_request* req, uint64_t* id);
/* Admit built nets, advance every lane by one step (its autotuned number
 * of intervals), retire finished nets.  *n_active (optional): nets running
 * after the step.  Returns immediately when nothing is running.  Not
 * reentrant: call it from one thread. */
int snn_server_step(snn_server* sv, int32_t* n_active);
/* State and counters of a request (thread-safe). */
int snn_server_poll(snn_server* sv, uint64_t id, snn_result* out);
/* Spikes (source, step) of a finished request that recorded them; *n is
 * the number recorded (SNN_E_OVERFLOW if above cap). */
int snn_server_spikes(snn_server* sv, uint64_t id, uint32_t* src, int32_t* t,
                      uint64_t cap, uint64_t* n);
/* Forget a finished request's result. */
int snn_server_release(snn_server* sv, uint64_t id);
/* Cancel a request (thread-safe).  A queued request leaves the queue at
 * once; one being built is destroyed when its build ends; a running one
 * leaves its batch at the next snn_server_step and is freed once the GPU
 * work already launched for it has completed.  Its state becomes
 * SNN_REQ_CANCELLED (no spikes or counters are kept) and its memory returns
 * to the budget.  SNN_E_STATE if it already finished, failed or was
 * cancelled; SNN_E_ARG for an unknown id. */
int snn_server_cancel(snn_server* sv, uint64_t id);
int snn_server_get_stats(snn_server* sv, snn_server_stats* out);
/* Stop the builder threads, free all nets; sv may be NULL. */
int snn_server_destroy(snn_server* sv);

#ifdef __cplusplus
}
#endif
#endif /* SNN_H */
