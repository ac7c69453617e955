"""Precision of the stored-weight formats against the FP64 oracle with the
UNROUNDED weights, at the benchmark sizes: the 112,500-neuron network
(1.27e9 synapses, fixed weights, delay 15 steps) with FP32 12-byte and BF16
8-byte records, and the 562,500-neuron network (6.3e9 synapses, BF16, weights
N(J, 0.1 J) / N(-5 J, 0.5 J), delays 10..20).

From one state of a running network, both sides deliver the same interval
spike list (8 Hz Bernoulli, emission steps [t0 - D, t0)) and then update one
interval [t0, t0 + D) with the same Poisson drive.  On a sample of targets:
  - ring buffer: |rb_gpu - rb_fp64| per cell, against the bound set by
    rounding each weight to its format (half an ulp: 2^-8 of |w| for BF16's
    8 significant bits, 2^-24 for FP32) plus the FP32 accumulation
    tolerance 1e-5 of the summed |w|;
  - membrane potential after the interval: |V_gpu - V_fp64|, against the
    ring-buffer error it can carry (at most the unit PSP peak, 4.46e-3 mV per
    pA of input error, the response being linear and its peak the largest
    value) plus 1e-4 mV of FP32 integration.
The measured errors are the per-config figures reported beside the speed of
each format."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import S, need_gpu, stream

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NM = O.Neuron()
NU_EXT_8HZ = 25757.293701171875
N_SAMPLE = 3000


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def precision_probe(wl, fmt, warm_steps=1000, seed=1):
    """Run the GPU net for warm_steps, then deliver one interval list and
    update one interval on both sides from the GPU's state.  Returns the
    error figures (dict) and the arrays for the bounds."""
    from paper_2109_12855_gb300 import snn
    from paper_2109_12855_gb300.tune import build_balanced
    D = wl.d_lo
    net, w_g = build_balanced(wl.n_e, wl.n_i, wl.k_e, wl.k_i, wl.d_lo, wl.d_hi,
                              fmt, wl.sd_rel, seed, stream(), psp_mv=wl.psp_mv,
                              g=wl.g, nu_ext=NU_EXT_8HZ)
    src, tt = W.bernoulli_spikes(wl.n, 0, D, 8.0, 0.1, seed=77)
    with net:
        snn.snn_set_drive(net.h, NU_EXT_8HZ, w_g)
        snn.snn_simulate(net.h, warm_steps)
        t0 = net.stats().t_now
        V, I, J, refr = net.read_state()
        snn.snn_clear_rb(net.h)
        net.deliver(src, (tt + t0 - D).astype(np.int32))
        rb_g = net.read_rb()[:, :N_SAMPLE].astype(np.float64)
        snn.snn_update(net.h, t0, D)
        snn.snn_discard_pending(net.h)
        V_g, _, _, refr_g = net.read_state()
        assert net.stats().error_flags == 0
    w_o = O.weight_for_psp(NM, wl.psp_mv)
    cp = O.Conn(wl.n_e, wl.n_i, wl.k_e, wl.k_i, w_o, -wl.g * w_o, wl.d_lo,
                wl.d_hi, seed + 1000, sd_e=wl.sd_rel * w_o,
                sd_i=wl.sd_rel * wl.g * w_o, wfmt=0)     # unrounded weights
    # the segments of every source onto the sampled targets [0, N_SAMPLE)
    store = O.build_fixed_indegree_targets(cp, 0, N_SAMPLE)
    rb_o, _, absw, _ = O.deliver_ref(store, S, src, tt + t0 - D)
    st = O.State(V.astype(np.float64), I.astype(np.float64),
                 J.astype(np.float64), refr.copy())
    O.update_range(NM, st, rb_o.copy(), 0, N_SAMPLE, t0, D, NU_EXT_8HZ, w_o,
                   seed)
    rb_o = rb_o[:, :N_SAMPLE]
    absw = absw[:, :N_SAMPLE]
    err = rb_g - rb_o
    touched = absw > 0
    same = refr_g[:N_SAMPLE] == st.refr[:N_SAMPLE]
    dv = np.abs(V_g[:N_SAMPLE].astype(np.float64) - st.V[:N_SAMPLE])
    fig = {"rb_max_abs_pa": float(np.abs(err).max()),
           "rb_rms_pa": float(np.sqrt(np.mean(err[touched] ** 2))),
           "rb_max_rel": float((np.abs(err)[touched] / absw[touched]).max()),
           "vm_max_abs_mv": float(dv[same].max()),
           "vm_rms_mv": float(np.sqrt(np.mean(dv[same] ** 2))),
           "spike_mismatch": int((~same).sum()),
           "cells": int(touched.sum())}
    return fig, err, absw, dv, same


@pytest.mark.parametrize("name,fmt", [("112500", 0), ("112500", 1),
                                      ("562500", 1)],
                         ids=["112500-fp32", "112500-bf16", "562500-bf16"])
def test_format_error_against_unrounded_fp64(name, fmt):
    wl = W.BALANCED_112500 if name == "112500" else W.BALANCED_562500
    fig, err, absw, dv, same = precision_probe(wl, fmt)
    u = 2.0 ** -8 if fmt == 1 else 2.0 ** -24
    bound = (u + 1e-5) * absw
    assert np.all(np.abs(err) <= bound), (fig, float((np.abs(err) - bound).max()))
    # the membrane bound: the whole interval's ring-buffer error of a neuron
    psp_per_pa = O.psp_peak(NM)[0]
    col_err = np.abs(err).sum(axis=0)
    assert np.all(dv[same] <= psp_per_pa * col_err[same] + 1e-4), fig
    assert fig["spike_mismatch"] <= 2, fig
    # the figures themselves: BF16 rounding is visible, FP32's is not
    if fmt == 1:
        assert 1e-4 < fig["rb_max_rel"] < 2.0 ** -8 + 1e-5, fig
    else:
        assert fig["rb_max_rel"] < 1e-5, fig
    print(name, fmt, fig)
