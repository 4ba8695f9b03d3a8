"""CUDA-graph capture of whole optimisation iterations.

Every launch of dgr_step / dgr_step_batched is asynchronous on the caller's
stream, allocates nothing and reads the step counter from device memory, so
one iteration can be captured once and replayed: one graph launch advances
every instance by one step.
"""
from __future__ import annotations

import torch

from . import dgr


class StepGraph:
    """Captures fn() (a sequence of dgr_* calls on torch's current stream)
    into a CUDA graph; replay() runs it again on the same device buffers."""

    def __init__(self, fn, warmup: int = 1):
        self.fn = fn
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            fn()
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()


def step_graph(prob, state, measured, loss, ws, warmup: int = 1) -> StepGraph:
    """Graph of one dgr_step (the warm-up steps advance the state)."""
    return StepGraph(lambda: dgr.dgr_step(prob, state, measured, loss, ws), warmup)


def batched_step_graph(probs, states, measured, losses, ws, warmup: int = 1) -> StepGraph:
    """Graph of one dgr_step_batched over all instances."""
    return StepGraph(lambda: dgr.dgr_step_batched(probs, states, measured, losses, ws), warmup)
