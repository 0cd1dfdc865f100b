"""ism_dataset_batch: the dataset step with host buffers (RIRs, convolution
and noise, Sec. II.A / III.A) over chunks of rooms with overlapped copies.
Its outputs equal the device entry points' bit for bit, for any chunking."""
import numpy as np
import pytest

from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_dataset_batch_matches_device_path(ism, precision):
    import torch
    rooms = wl.ragged_batch(11, seed=404, rt_hi=0.25)
    srcs = wl.sources(rooms, 0.2, seed=405)
    snr = wl.snrs(11, seed=406)
    snr[3] = np.nan  # one room without noise
    lens = [len(s) for s in srcs]
    src_cat = np.concatenate(srcs)
    # device path
    h = ism.rir_batch(rooms)
    jobs, ylen = ism.conv_jobs([len(r["mics"]) for r in rooms], [r["rir_len"] for r in rooms], lens,
                               snr_db=snr, noise_ids=np.arange(11) + 500)
    y = torch.empty(ylen, device="cuda")
    ism.convolve_batch(jobs, h, torch.from_numpy(src_cat).cuda(), y, seed=8, precision=precision)
    torch.cuda.synchronize()
    y_ref, h_ref = y.cpu(), h.cpu()
    src_pin = torch.from_numpy(src_cat).pin_memory()
    for chunk in (0, 1, 3, 11):
        y_host = torch.full((ylen,), float("nan")).pin_memory()
        h_host = torch.full((h_ref.numel(),), float("nan")).pin_memory()
        ism.dataset_batch(rooms, src_pin, lens, y_host, snr_db=snr, seed=8, noise_id_base=500,
                          precision=precision, h_host=h_host, chunk_rooms=chunk)
        assert torch.equal(y_host, y_ref), chunk
        assert torch.equal(h_host, h_ref), chunk
    # pageable host buffers work too
    y_np = np.zeros(ylen, np.float32)
    ism.dataset_batch(rooms, src_cat, lens, y_np, snr_db=snr, seed=8, noise_id_base=500,
                      precision=precision)
    np.testing.assert_array_equal(y_np, y_ref.numpy())


def test_dataset_batch_tile_round_chunks(ism):
    """Enough 8-mic rooms (160 rooms, 1 s sources, 8192-sample RIRs: 960
    convolution tiles) for the automatic split to cut chunks at whole rounds
    of tiles over the SMs: the outputs equal one chunk's bit for bit."""
    import torch
    n = 160
    rooms = wl.room_batch(n, seed=407)
    srcs = wl.sources(rooms, 1.0, seed=408)
    snr = wl.snrs(n, seed=409)
    lens = [len(s) for s in srcs]
    src_pin = torch.from_numpy(np.concatenate(srcs)).pin_memory()
    ylen = sum(8 * (t + r["rir_len"] - 1) for t, r in zip(lens, rooms))
    outs = []
    for chunk in (0, n):
        y_host = torch.full((ylen,), float("nan")).pin_memory()
        ism.dataset_batch(rooms, src_pin, lens, y_host, snr_db=snr, seed=9, noise_id_base=7,
                          precision=1, chunk_rooms=chunk)
        outs.append(y_host)
    assert not torch.isnan(outs[0]).any()
    assert torch.equal(outs[0], outs[1])
