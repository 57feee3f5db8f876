"""Host-resident holograms through one plan, with the copies hidden.

A caller whose holograms and results live in host memory pays a 8 N^2-byte
host->device copy and a device->host copy of the view per reconstruction.
HostPipeline overlaps them with the GPU work: hologram i+1 is copied in on
one stream and view i-1 copied out on another while view i is reconstructed
on the caller's stream, with two device staging buffers each way.  Every
step still runs the whole path (load of the new hologram's spectrum, stretch,
Fresnel transform, remap) through the C ABI; only the copies move.

Host buffers should be pinned (torch ``pin_memory=True``) for the copies to
be asynchronous.  ``h_out`` of a submitted step is valid once the caller's
stream has passed ``drain()`` (or after a device synchronize).
"""
from __future__ import annotations


class HostPipeline:
    def __init__(self, plan, view, stream=None):
        import torch
        self.torch = torch
        self.plan, self.view = plan, view
        self.main = stream if stream is not None else torch.cuda.current_stream()
        self.s_in, self.s_out = torch.cuda.Stream(), torch.cuda.Stream()
        shape = (plan.ny, plan.nx)
        self.d_in = [torch.empty(shape, dtype=torch.complex64, device="cuda") for _ in range(2)]
        self.d_out = [plan.output_like(view) for _ in range(2)]
        E = torch.cuda.Event
        self.ev_in = [E(), E()]      # hologram k on the device
        self.ev_load = [E(), E()]    # spectrum of hologram k cached: staging buffer k free
        self.ev_rec = [E(), E()]     # view k reconstructed
        self.ev_out = [E(), E()]     # view k copied out: output buffer k free
        self.i = 0

    def begin(self):
        """Order the copy streams after the work already on the caller's stream."""
        self.s_in.wait_stream(self.main)
        self.s_out.wait_stream(self.main)

    def submit(self, h_holo, h_out):
        """Enqueue one step: copy h_holo in, reconstruct, copy the view to h_out."""
        torch, k = self.torch, self.i % 2
        if self.i >= 2:
            self.s_in.wait_event(self.ev_load[k])
        with torch.cuda.stream(self.s_in):
            self.d_in[k].copy_(h_holo, non_blocking=True)
            self.ev_in[k].record(self.s_in)
        self.main.wait_event(self.ev_in[k])
        self.plan.load(self.d_in[k], stream=self.main)
        self.ev_load[k].record(self.main)
        if self.i >= 2:
            self.main.wait_event(self.ev_out[k])
        self.plan.reconstruct(self.view, self.d_out[k], stream=self.main)
        self.ev_rec[k].record(self.main)
        self.s_out.wait_event(self.ev_rec[k])
        with torch.cuda.stream(self.s_out):
            h_out.copy_(self.d_out[k], non_blocking=True)
            self.ev_out[k].record(self.s_out)
        self.i += 1

    def drain(self):
        """Make the caller's stream wait for every copy-out submitted so far."""
        for k in range(min(self.i, 2)):
            self.main.wait_event(self.ev_out[k])
