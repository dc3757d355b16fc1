"""Seeded synthetic graph generators shared by the tests, the bench and the oracle's fixtures.

This package holds no part of the truss method's arithmetic: it only draws raw
undirected edge lists (``src``, ``dst`` int32 arrays) from named random-graph
models.  Normalisation (self-loops, duplicates, reverse pairs) is the job of the
code under test, so several generators deliberately return raw pairs.
"""

from .generators import (  # noqa: F401
    CONFIG_SEED_BASE,
    GraphSpec,
    barabasi_albert,
    batch_graph,
    batch_graphs,
    batch_params,
    config_graph,
    dcsbm,
    erdos_renyi_gnm,
    rmat,
    served_requests,
    small_corpus,
)
