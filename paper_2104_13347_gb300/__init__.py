"""GB300-native image-source RIR synthesis and multichannel convolution.

The dataset-generation hot path of arXiv 2104.13347 (Sec. II.A): shoebox
room impulse responses from the image-source method with fractional delays,
then batch convolution of source signals with the RIRs into microphone
pressure, with additive noise at a chosen SNR (Sec. III.A), and the noisy
multichannel training frames cut from those signals (Sec. II.B / III.A).  The compute runs
in libism.so (hand-written CUDA for sm_103a) behind the C ABI of
include/ism.h; this package is its Python binding.

    import paper_2104_13347_gb300 as ism
    h = ism.rir_batch(rooms)            # float32 CUDA tensor, packed RIRs
"""
from ._lib import (BF16X3, F32, FD_HANN_SINC, FD_LAGRANGE, INJECT_CONV_WAIT, INJECT_SERVE_ALLOC, RIR_DIRECT,  # noqa
                   RIR_SPARSE, IsmError, PreparedRooms, check, conv_jobs, convolve_batch,
                   dataset_batch, debug_bounds, debug_inject, frame_jobs, frames_batch, last_error, load,
                   make_rooms, Plan, rir_batch, rir_batch_noalloc, rir_batch_size, rir_filter_terms,
                   rir_tuned_window, Server, stream_status, WINDOW_TUNE)

__all__ = ["load", "rir_batch", "rir_batch_size", "rir_batch_noalloc", "convolve_batch",
           "conv_jobs", "dataset_batch", "frame_jobs", "frames_batch", "IsmError", "F32", "BF16X3", "FD_HANN_SINC", "FD_LAGRANGE", "RIR_SPARSE",
           "RIR_DIRECT", "last_error", "check", "make_rooms", "PreparedRooms", "rir_filter_terms", "Server",
           "stream_status", "debug_inject", "debug_bounds", "INJECT_CONV_WAIT", "INJECT_SERVE_ALLOC", "rir_tuned_window",
           "WINDOW_TUNE", "Plan"]
