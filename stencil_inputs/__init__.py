"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws numbers: grids, coefficient cubes and job mixes.  It
holds none of the stencil method's arithmetic, so both the CUDA path's tests
and the FP64 oracle can use it without sharing any of the computation.

Every generator is numpy ``PCG64`` seeded with ``BASE_SEED + workload index``
(plus a per-draw offset where one workload needs several draws).  Grids are
float32, x fastest, C-contiguous.

The paper evaluates synthetic stencil shapes only (Sec. 4.1: 1-D r = 1, 2 and
2-D star / box r = 1..3 on 10240^2); these generators produce the same kind
of inputs at the sizes of the workloads below.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20250622

STAR, BOX = "star", "box"


def rng(workload: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + workload + 1000 * sub))


def grid(shape, low: float, high: float, gen: np.random.Generator) -> np.ndarray:
    """float32 grid, uniform on [low, high)."""
    return gen.uniform(low, high, size=tuple(shape)).astype(np.float32)


def star_mask(ndim: int, r: int) -> np.ndarray:
    """Offsets of a star stencil inside the (2r+1)^d cube (on one axis only)."""
    side = 2 * r + 1
    m = np.zeros((side,) * ndim, dtype=bool)
    centre = (r,) * ndim
    for ax in range(ndim):
        for o in range(side):
            idx = list(centre)
            idx[ax] = o
            m[tuple(idx)] = True
    return m


def normalised_coeffs(ndim: int, r: int, shape: str, gen: np.random.Generator) -> np.ndarray:
    """Uniform[0,1) coefficients on the stencil's offsets, scaled to sum 1
    (in float64, then stored as float32); off-stencil entries are 0."""
    side = 2 * r + 1
    w = gen.uniform(0.0, 1.0, size=(side,) * ndim)
    if shape == STAR:
        w = np.where(star_mask(ndim, r), w, 0.0)
    elif shape != BOX:
        raise ValueError("shape must be 'star' or 'box'")
    w = w / w.sum()
    return w.astype(np.float32)


def heat2d_coeffs() -> np.ndarray:
    """5-point heat stencil: centre 0.6, each neighbour 0.1 (float32)."""
    w = np.zeros((3, 3), dtype=np.float32)
    w[1, 1] = 0.6
    w[0, 1] = w[2, 1] = w[1, 0] = w[1, 2] = 0.1
    return w


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    ndim: int
    extents: tuple
    shape: str
    r: int
    steps: int
    low: float
    high: float
    index: int


HEAT2D_512 = Workload("heat2d-star-r1-512^2", 2, (512, 512), STAR, 1, 10, 0.0, 1.0, 0)
BOX2D_R3_8192 = Workload("box2d-r3-8192^2", 2, (8192, 8192), BOX, 3, 100, -1.0, 1.0, 1)
HEAT3D_512 = Workload("heat3d-star-r1-512^3", 3, (512, 512, 512), STAR, 1, 50, 0.0, 1.0, 2)
BOX3D_512 = Workload("box3d-r1-512^3", 3, (512, 512, 512), BOX, 1, 50, 0.0, 1.0, 2)


def workload_inputs(wl: Workload, extents=None):
    """(grid, coefficients) for a workload; ``extents`` overrides the size
    (same distributions, same seeds) for scaled-down parity cases."""
    ext = tuple(extents) if extents is not None else wl.extents
    g = rng(wl.index, 0)
    u0 = grid(ext, wl.low, wl.high, g)
    if wl is HEAT2D_512 or wl.name.startswith("heat2d"):
        w = heat2d_coeffs()
    else:
        w = normalised_coeffs(wl.ndim, wl.r, wl.shape, rng(wl.index, 1 if wl.shape == BOX else 2))
    return u0, w


@dataclasses.dataclass(frozen=True)
class Job:
    ndim: int
    extents: tuple
    shape: str
    r: int
    steps: int
    seed: int
    err_target: float = 1e-3
    arrival_s: float = 0.0


def log_uniform_int(gen: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(gen.uniform(math.log(lo), math.log(hi)))))


def batched_jobs(n: int = 64, workload: int = 3) -> list[Job]:
    """Batched mix: 2-D grids, each side log-uniform in [256, 4096] (drawn
    independently per axis), shape uniform in {star, box}, r uniform in
    {1, 2, 3}, steps uniform in [10, 200]."""
    g = rng(workload, 0)
    jobs = []
    for i in range(n):
        ny = log_uniform_int(g, 256, 4096)
        nx = log_uniform_int(g, 256, 4096)
        shape = STAR if g.integers(0, 2) == 0 else BOX
        r = int(g.integers(1, 4))
        steps = int(g.integers(10, 201))
        jobs.append(Job(2, (ny, nx), shape, r, steps, BASE_SEED + workload + 7919 * (i + 1)))
    return jobs


def batched_small_jobs(n: int = 256, workload: int = 5) -> list[Job]:
    """Small-grid batch: 2-D grids, each side log-uniform in [32, 255] (drawn
    independently per axis, so every grid has fewer than 2^16 points), shape
    uniform in {star, box}, r uniform in {1, 2, 3}, steps uniform in
    [10, 200]."""
    g = rng(workload, 0)
    jobs = []
    for i in range(n):
        ny = log_uniform_int(g, 32, 255)
        nx = log_uniform_int(g, 32, 255)
        shape = STAR if g.integers(0, 2) == 0 else BOX
        r = int(g.integers(1, 4))
        steps = int(g.integers(10, 201))
        jobs.append(Job(2, (ny, nx), shape, r, steps, BASE_SEED + workload + 7919 * (i + 1)))
    return jobs


def serving_arrivals(n: int = 2000, rate_per_s: float = 200.0, workload: int = 4) -> list[Job]:
    """Serving mix: Poisson arrivals; half 2-D (side log-uniform 256-8192),
    half 3-D (side log-uniform 64-512); r uniform 1..3; shape uniform
    {star, box}; steps uniform 10..500; error target 1e-3 or 1e-5."""
    g = rng(workload, 0)
    t = 0.0
    jobs = []
    for i in range(n):
        t += float(g.exponential(1.0 / rate_per_s))
        if g.integers(0, 2) == 0:
            side = log_uniform_int(g, 256, 8192)
            ndim, ext = 2, (side, side)
        else:
            side = log_uniform_int(g, 64, 512)
            ndim, ext = 3, (side, side, side)
        r = int(g.integers(1, 4))
        shape = STAR if g.integers(0, 2) == 0 else BOX
        steps = int(g.integers(10, 501))
        err = 1e-3 if g.integers(0, 2) == 0 else 1e-5
        jobs.append(Job(ndim, ext, shape, r, steps, BASE_SEED + workload + 7919 * (i + 1), err, t))
    return jobs


def serving_grid_pool(jobs, workload: int = 4) -> np.ndarray:
    """One U[0,1) float32 buffer as large as the largest job of `jobs`; each
    serving job's grid is its prefix, reshaped (drawing every job's grid of up
    to 512^3 points on the host would take longer than serving it)."""
    n = max(int(np.prod(j.extents)) for j in jobs)
    return grid((n,), 0.0, 1.0, rng(workload, 7))


def serving_job_coeffs(job: Job) -> np.ndarray:
    """The serving job's coefficients: normalised random from its own seed."""
    return normalised_coeffs(job.ndim, job.r, job.shape, np.random.Generator(np.random.PCG64(job.seed + 1)))


def job_inputs(job: Job):
    g = np.random.Generator(np.random.PCG64(job.seed))
    u0 = grid(job.extents, 0.0, 1.0, g)
    w = normalised_coeffs(job.ndim, job.r, job.shape, g)
    return u0, w
