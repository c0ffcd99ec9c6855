"""Batching of many clients' uneven query batches (Sec. 3: batch inference fills
the SIMD slots; Sec. 4.1: one score ciphertext per packed group).

Requests are packed back to back into one query space, so groups of `cap` queries
may hold several clients' queries; the encrypted model is then streamed once for
all groups.  The device work of one packed step is replayed from a CUDA graph
captured per group count G: the packed features are copied into a static buffer
whose rows past the last request are zero, which changes no real query's result
(a zero feature row only fills unused slots), so one graph per G serves every mix
of requests that needs G groups.
"""
import math

import torch

from . import ephdc as E


class PackedBatch:
    """Where each request's queries sit in the packed query space."""

    def __init__(self, sizes, cap):
        self.sizes = [int(b) for b in sizes]
        self.offsets = []
        off = 0
        for b in self.sizes:
            self.offsets.append(off)
            off += b
        self.total = off
        self.cap = cap
        self.groups = max(1, math.ceil(off / cap))

    def rows(self, r):
        return slice(self.offsets[r], self.offsets[r] + self.sizes[r])


class GraphedPipeline:
    """Client path for packed requests, replayed from per-G CUDA graphs."""

    def __init__(self, ctx, Wt, model, gk, max_groups=None, use_graphs=True):
        self.ctx, self.Wt, self.model, self.gk = ctx, Wt, model, gk
        self.cap = ctx.cap
        self.max_groups = max_groups or max(1, ctx.max_batch // ctx.cap)
        rows = self.max_groups * self.cap
        if rows > ctx.max_batch:
            raise ValueError("max_groups * cap exceeds the context's max_batch")
        dev = ctx.device
        self.X = torch.zeros((rows, ctx.F), dtype=torch.int8, device=dev)
        self.ct_words = ctx.Kp * 2 * ctx.L * ctx.n
        self.out = torch.zeros(self.max_groups * self.ct_words, dtype=torch.int32, device=dev)
        self.use_graphs = use_graphs
        self.graphs = {}
        self.stream = torch.cuda.Stream(device=dev)

    def _launch(self, G):
        B = G * self.cap
        self.ctx.infer(self.X[:B], self.Wt, self.model, self.gk,
                       out=self.out[:G * self.ct_words])

    def graph(self, G):
        if G not in self.graphs:
            with torch.cuda.stream(self.stream):
                self._launch(G)  # warm-up outside capture (tables, attributes)
            self.stream.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=self.stream):
                self._launch(G)
            self.graphs[G] = g
        return self.graphs[G]

    def pack(self, Xs):
        pb = PackedBatch([x.shape[0] for x in Xs], self.cap)
        if pb.groups > self.max_groups:
            raise ValueError("packed batch needs %d groups, at most %d" % (pb.groups,
                                                                           self.max_groups))
        for r, x in enumerate(Xs):
            if pb.sizes[r]:
                self.X[pb.rows(r)].copy_(x, non_blocking=True)
        end = pb.groups * self.cap
        if pb.total < end:
            self.X[pb.total:end].zero_()
        return pb

    def run(self, Xs):
        """Runs one packed step on the current stream; returns (score ciphertexts of
        the G groups, PackedBatch)."""
        pb = self.pack(Xs)
        if self.use_graphs:
            g = self.graph(pb.groups)
            self.stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(self.stream):
                g.replay()
            torch.cuda.current_stream().wait_stream(self.stream)
        else:
            self._launch(pb.groups)
        return self.out[:pb.groups * self.ct_words], pb

    def launch(self, Xs, stream):
        """Packs and runs one step entirely on `stream`, with no synchronisation with
        other streams (the graph for the step's group count must already exist or is
        captured first).  Returns (score ciphertexts of the G groups, PackedBatch)."""
        if self.use_graphs:
            pb = PackedBatch([x.shape[0] for x in Xs], self.cap)
            self.graph(pb.groups)
        with torch.cuda.stream(stream):
            pb = self.pack(Xs)
            if self.use_graphs:
                self.graphs[pb.groups].replay()
            else:
                self._launch(pb.groups)
        return self.out[:pb.groups * self.ct_words], pb
