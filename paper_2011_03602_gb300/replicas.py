"""Serving replicas with one process per GPU.

Requests are independent, so the replicas share nothing but the routing
figures: in each routing round every rank contributes its server's free
device bytes and requests in flight (one all-gather of two integers per
rank), and every rank then runs the library's routing rule
(oo_route_batch: most free bytes among replicas with room, ties to fewer in
flight, then the lower rank) over the same request list, so all ranks agree
on the owner of every request without exchanging the requests' data.  Each
rank serves the requests it owns on its own GPU.  This suits a front end
that delivers every request to every rank (a broadcast feed, or a
deterministic request generator as in the tests); with one process holding
several GPUs, oo_router_* routes in-process instead.
"""
import numpy as np
import torch
import torch.distributed as dist

from . import oo


def gather_figures(free_bytes, in_flight, group=None):
    """-> (free bytes per rank, requests in flight per rank), rank order."""
    t = torch.tensor([int(free_bytes), int(in_flight)], dtype=torch.int64)
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(out, t, group=group)
    return [int(o[0]) for o in out], [int(o[1]) for o in out]


def route_round(needs, free_bytes, in_flight, group=None):
    """Owners (rank per request) of one routing round; every rank calls it
    with the same `needs` (footprint bytes per request, oo_serve_footprint)
    and its own figures, and gets the same answer."""
    f, q = gather_figures(free_bytes, in_flight, group)
    return oo.oo_route_batch(f, q, needs)


def serve_round(ctx, requests, group=None, timeout_ms=600000):
    """Route a round of requests [(kind, kwargs)] (the same list on every
    rank) and serve the ones this rank owns on its serving context `ctx`.
    Returns the owners and {request index: latency ms} of this rank's."""
    rank = dist.get_rank(group)
    reqs = [oo.serve_request(k, **kw) for k, kw in requests]
    needs = [oo.oo_serve_footprint(r) for r in reqs]
    st = oo.oo_serve_stats(ctx)
    owners = route_round(needs, st["device_free_bytes"], st["queued"] + st["running"], group)
    mine = [(i, oo.oo_submit(ctx, reqs[i])) for i in range(len(reqs)) if owners[i] == rank]
    return owners, {i: oo.oo_wait(ctx, t, timeout_ms) for i, t in mine}


__all__ = ["gather_figures", "route_round", "serve_round"]
