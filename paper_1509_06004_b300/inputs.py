"""Seeded synthetic inputs for the grid min-cut workloads.

This module only builds input arrays: a synthetic image, the int32 pairwise
capacities of its 4-connected grid graph, the terminal capacities of each
(image, foreground seed) instance and the increasing lambda schedule.  It holds
none of the max-flow arithmetic and imports nothing else from this package, so
both the CPU oracle (tests) and the CUDA path are fed from it.

The graph follows Section 2 of the paper (a node per pixel, terminal edges to
the source s and the sink t, pairwise edges to the up/down/left/right
neighbours), the seeds follow Section 2.1 (foreground seeds on a regular grid
or at random interior spots, background seeds on the image border, seed pixels
"frozen" to their side) and the lambda schedule is the preset, logarithmically
spaced list of Section 2.1.

Capacity recipe (one image I with values in [0, 1]):
  w_h[y, x] = floor(1000 * exp(-(I[y,x] - I[y,x+1])^2 / (2 * 0.1^2))), 0 on the last column
  w_v[y, x] = floor(1000 * exp(-(I[y,x] - I[y+1,x])^2 / (2 * 0.1^2))), 0 on the last row
  seed pixels:   cs = INF, ct = 0              (src0 = INF, slope = 0, sink = 0)
  border pixels: cs = 0,   ct = INF            (src0 = 0,   slope = 0, sink = INF)
  other pixels:  cs = lambda, ct = rint(1000 * |I - mean(I over the seed)|)
                                               (src0 = 0,   slope = 1, sink = t_p)
so the source capacity of pixel p at parameter lambda is src0[p] + slope[p] * lambda.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

INF = 1 << 30          # "infinite" terminal capacity; int32 headroom is 2^31 - 1
W_SCALE = 1000.0       # pairwise capacity scale
W_SIGMA = 0.1          # contrast scale of the pairwise term
SEED_SIZE = 5          # foreground seeds are 5x5 squares


# ----------------------------------------------------------------------------
# images, capacities, seeds, schedules
# ----------------------------------------------------------------------------

def make_image(H: int, W: int, n_ellipses: int, sigma: float,
               rng: np.random.Generator) -> np.ndarray:
    """Background 0 plus ``n_ellipses`` filled ellipses of constant intensity
    U(0,1), later ones painted over earlier ones, plus N(0, sigma^2) noise,
    clipped to [0, 1].  Draw order per ellipse: intensity, centre y, centre x,
    semi-axis a (rows), semi-axis b (cols), angle; then the noise field."""
    img = np.zeros((H, W), dtype=np.float64)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_ellipses):
        val = rng.uniform(0.0, 1.0)
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        a = rng.uniform(0.1, 0.4) * H
        b = rng.uniform(0.1, 0.4) * W
        th = rng.uniform(0.0, np.pi)
        dy, dx = yy - cy, xx - cx
        u = dy * np.cos(th) + dx * np.sin(th)
        v = -dy * np.sin(th) + dx * np.cos(th)
        img[(u / a) ** 2 + (v / b) ** 2 <= 1.0] = val
    img += rng.normal(0.0, sigma, size=(H, W))
    return np.clip(img, 0.0, 1.0)


def pairwise_caps(img: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric contrast-sensitive pairwise capacities (int32, shape H x W).
    ``w_h[y, x]`` joins (y, x)-(y, x+1); ``w_v[y, x]`` joins (y, x)-(y+1, x)."""
    H, W = img.shape
    w_h = np.zeros((H, W), dtype=np.int32)
    w_v = np.zeros((H, W), dtype=np.int32)
    k = 2.0 * W_SIGMA * W_SIGMA
    w_h[:, :-1] = np.floor(W_SCALE * np.exp(-(img[:, :-1] - img[:, 1:]) ** 2 / k))
    w_v[:-1, :] = np.floor(W_SCALE * np.exp(-(img[:-1, :] - img[1:, :]) ** 2 / k))
    return w_h, w_v


def border_mask(H: int, W: int) -> np.ndarray:
    m = np.zeros((H, W), dtype=bool)
    m[0, :] = m[-1, :] = True
    m[:, 0] = m[:, -1] = True
    return m


def seed_square(H: int, W: int, y0: int, x0: int, size: int = SEED_SIZE) -> np.ndarray:
    m = np.zeros((H, W), dtype=bool)
    m[y0:y0 + size, x0:x0 + size] = True
    return m


def random_seed_origin(H: int, W: int, rng: np.random.Generator) -> tuple[int, int]:
    """Top-left corner of a 5x5 seed, uniform over [1, H-6] x [1, W-6] so the
    square never touches the one-pixel background border."""
    y0 = int(rng.integers(1, H - SEED_SIZE - 1 + 1))
    x0 = int(rng.integers(1, W - SEED_SIZE - 1 + 1))
    return y0, x0


def grid_seed_origins(H: int, W: int, n: int = 5) -> list[tuple[int, int]]:
    """n x n regular grid of seed centres c = floor((i + 0.5) * size / n),
    squares [c-2, c+2]^2 (returned as top-left corners)."""
    out = []
    for i in range(n):
        for j in range(n):
            cy = int(np.floor((i + 0.5) * H / n))
            cx = int(np.floor((j + 0.5) * W / n))
            out.append((cy - SEED_SIZE // 2, cx - SEED_SIZE // 2))
    return out


def terminals(img: np.ndarray, seed: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(src0, slope, sink) int32 planes for one (image, seed) instance."""
    H, W = img.shape
    border = border_mask(H, W)
    assert not (border & seed).any(), "seed touches the background border"
    mean_seed = float(img[seed].mean())
    src0 = np.zeros((H, W), dtype=np.int32)
    slope = np.ones((H, W), dtype=np.int32)
    sink = np.rint(W_SCALE * np.abs(img - mean_seed)).astype(np.int32)
    src0[seed] = INF
    slope[seed] = 0
    sink[seed] = 0
    src0[border] = 0
    slope[border] = 0
    sink[border] = INF
    return src0, slope, sink


def lambda_schedule(m: int, lo: float, hi: float) -> np.ndarray:
    """rint(lo * (hi/lo)^(k/(m-1))), k = 0..m-1, strictly increasing int32."""
    if m == 1:
        return np.array([int(np.rint(lo))], dtype=np.int32)
    k = np.arange(m, dtype=np.float64)
    lam = np.rint(lo * (hi / lo) ** (k / (m - 1))).astype(np.int64)
    assert np.all(np.diff(lam) > 0), "lambda schedule not strictly increasing"
    return lam.astype(np.int32)


# ----------------------------------------------------------------------------
# workload containers
# ----------------------------------------------------------------------------

@dataclass
class Image:
    H: int
    W: int
    w_h: np.ndarray          # int32 [H, W]
    w_v: np.ndarray          # int32 [H, W]
    img: np.ndarray | None = None


@dataclass
class Instance:
    image: int               # index into Workload.images
    src0: np.ndarray         # int32 [H, W]
    slope: np.ndarray        # int32 [H, W]
    sink: np.ndarray         # int32 [H, W]
    lambdas: np.ndarray      # int32 [m], strictly increasing
    seed_origin: tuple[int, int] = (0, 0)
    # for a piece of a split schedule: (index of the instance it was cut from,
    # int array of the positions of its lambdas in that instance's schedule)
    origin: tuple | None = None
    # for a forked piece: (index of the parent instance in the same workload,
    # the parent's step after which this piece starts from its state)
    fork: tuple | None = None


@dataclass
class Workload:
    name: str
    images: list[Image] = field(default_factory=list)
    instances: list[Instance] = field(default_factory=list)

    @property
    def n_solves(self) -> int:
        return sum(len(i.lambdas) for i in self.instances)

    @property
    def pixel_solves(self) -> int:
        return sum(self.images[i.image].H * self.images[i.image].W * len(i.lambdas)
                   for i in self.instances)

    def _piece(self, i: int, inst: Instance, idx) -> Instance:
        idx = np.asarray(idx, dtype=np.int64)
        base = inst.origin
        # a piece of a piece keeps pointing at the original schedule
        o = (i, idx) if base is None else (base[0], base[1][idx])
        return Instance(inst.image, inst.src0, inst.slope, inst.sink, inst.lambdas[idx].astype(np.int32),
                        inst.seed_origin, o)

    def split_segments(self, segments: int) -> "Workload":
        """Every instance's schedule cut into ``segments`` consecutive pieces of
        equal length, each its own instance (warm-started inside a piece, cold
        at its first lambda).  segments = 1 is the workload itself; segments =
        schedule length is split_lambdas()."""
        out = Workload(self.name + (f"/seg{segments}" if segments > 1 else ""), list(self.images), [])
        for i, inst in enumerate(self.instances):
            m = len(inst.lambdas)
            if m % segments:
                raise ValueError(f"{segments} segments do not divide a schedule of {m}")
            for part in np.split(np.arange(m), segments):
                out.instances.append(self._piece(i, inst, part))
        return out

    def split_pieces(self, lengths) -> "Workload":
        """Every instance's schedule cut into consecutive pieces of the given
        lengths (summing to the schedule length), each its own instance,
        warm-started inside a piece and cold at its first lambda.  Unlike
        split_segments the pieces may differ in length."""
        lengths = [int(x) for x in lengths]
        if min(lengths) < 1:
            raise ValueError("pieces need at least one lambda")
        out = Workload(self.name + "/pieces" + "-".join(map(str, lengths)), list(self.images), [])
        for i, inst in enumerate(self.instances):
            if sum(lengths) != len(inst.lambdas):
                raise ValueError(f"pieces {lengths} do not cover a schedule of {len(inst.lambdas)}")
            for part in np.split(np.arange(len(inst.lambdas)), np.cumsum(lengths)[:-1]):
                out.instances.append(self._piece(i, inst, part))
        return out

    def split_forked(self, segments: int, lead: int) -> "Workload":
        """Every instance's schedule cut into ``segments`` consecutive pieces
        (as split_segments), each piece after the first FORKED from the one
        before: it starts from that piece's state once the piece has
        certified its step (length - 1 - lead), instead of cold.  lead = 0
        forks after the previous piece's last step (a chain, as one piece);
        a larger lead starts the next piece that many steps earlier, so the
        two run side by side, the new piece warm-started from a lambda
        ``lead + 1`` steps below its first."""
        if lead < 0:
            raise ValueError("lead >= 0")
        out = self.split_segments(segments)
        out.name = self.name + f"/fork{segments}x{lead}"
        first = 0
        for inst in self.instances:
            n = segments
            for j in range(1, n):
                prev = out.instances[first + j - 1]
                step = max(0, len(prev.lambdas) - 1 - lead)
                out.instances[first + j].fork = (first + j - 1, step)
            first += n
        return out

    def split_interleaved(self, stride: int) -> "Workload":
        """Every instance's schedule dealt round-robin into ``stride`` pieces:
        piece j holds lambda_j, lambda_{j+stride}, lambda_{j+2*stride}, ...
        Each piece starts cold at one of the schedule's ``stride`` smallest
        lambdas and is warm-started along its own (coarser, still
        nondecreasing) schedule, so neighbouring lambdas of one seed are solved
        side by side.  stride = 1 is the workload itself."""
        out = Workload(self.name + (f"/ilv{stride}" if stride > 1 else ""), list(self.images), [])
        for i, inst in enumerate(self.instances):
            m = len(inst.lambdas)
            if not 1 <= stride <= m:
                raise ValueError(f"stride {stride} outside [1, {m}]")
            for j in range(stride):
                out.instances.append(self._piece(i, inst, np.arange(j, m, stride)))
        return out

    def split_lambdas(self) -> "Workload":
        """The same solves with every (instance, lambda) as its own one-lambda
        instance (the lambda-concurrent form: no warm start between lambdas)."""
        out = Workload(self.name + "/lambda-split", list(self.images), [])
        for i, inst in enumerate(self.instances):
            for k in range(len(inst.lambdas)):
                out.instances.append(self._piece(i, inst, [k]))
        return out

    def gather(self, results, n_instances: int | None = None):
        """Results of a split workload ([(flows [m_i], masks [m_i, H, W])] per
        piece, in this workload's instance order) put back per original
        instance: a list of (flows [m], masks [m, H, W]).  Pieces without an
        origin are their own original instance.  Every lambda of every
        original instance must be covered exactly once."""
        groups: dict[int, list] = {}
        for j, (inst, (f, m)) in enumerate(zip(self.instances, results)):
            oi, idx = inst.origin if inst.origin is not None else (j, np.arange(len(inst.lambdas)))
            groups.setdefault(oi, []).append((idx, f, m))
        n = n_instances if n_instances is not None else max(groups) + 1
        out = []
        for oi in range(n):
            parts = groups[oi]
            m_len = sum(len(idx) for idx, _, _ in parts)
            f0, mk0 = parts[0][1], parts[0][2]
            flows = np.zeros(m_len, dtype=np.asarray(f0).dtype)
            masks = np.zeros((m_len,) + mk0.shape[1:], dtype=mk0.dtype)
            seen = np.zeros(m_len, dtype=bool)
            for idx, f, mk in parts:
                if seen[idx].any():
                    raise ValueError(f"lambda covered twice in instance {oi}")
                seen[idx] = True
                flows[idx] = f
                masks[idx] = mk
            if not seen.all():
                raise ValueError(f"lambda not covered in instance {oi}")
            out.append((flows, masks))
        return out


def _image(H: int, W: int, n_ell: int, sigma: float, rng: np.random.Generator) -> Image:
    img = make_image(H, W, n_ell, sigma, rng)
    w_h, w_v = pairwise_caps(img)
    return Image(H, W, w_h, w_v, img)


def _instance(wl: Workload, image: int, y0: int, x0: int, lambdas: np.ndarray) -> None:
    im = wl.images[image]
    seed = seed_square(im.H, im.W, y0, x0)
    src0, slope, sink = terminals(im.img, seed)
    wl.instances.append(Instance(image, src0, slope, sink, lambdas, (y0, x0)))


# ----------------------------------------------------------------------------
# the five workload shapes
# ----------------------------------------------------------------------------

def single_maxflow_64(seed: int = 0) -> Workload:
    """One 64x64 grid, 3 ellipses, sigma 0.05, one random 5x5 seed, lambda 300."""
    rng = np.random.default_rng(seed)
    wl = Workload("single-64x64")
    wl.images.append(_image(64, 64, 3, 0.05, rng))
    y0, x0 = random_seed_origin(64, 64, rng)
    _instance(wl, 0, y0, x0, np.array([300], dtype=np.int32))
    return wl


def parametric_320x240(seed: int = 0, n_lambda: int = 20) -> Workload:
    """One 320x240 grid (W=320, H=240), one random seed, 20 lambdas in [10, 5000]."""
    rng = np.random.default_rng(seed)
    wl = Workload("parametric-320x240")
    wl.images.append(_image(240, 320, 3, 0.05, rng))
    y0, x0 = random_seed_origin(240, 320, rng)
    _instance(wl, 0, y0, x0, lambda_schedule(n_lambda, 10, 5000))
    return wl


def supergraph_480x320(seed: int = 0, n_lambda: int = 20, grid: int = 5) -> Workload:
    """One 480x320 image (W=480, H=320), 25 seeds on a 5x5 grid, 20 lambdas in
    [10, 5000]: 500 parametric solves."""
    rng = np.random.default_rng(seed)
    wl = Workload("supergraph-480x320")
    wl.images.append(_image(320, 480, 3, 0.05, rng))
    lam = lambda_schedule(n_lambda, 10, 5000)
    for (y0, x0) in grid_seed_origins(320, 480, grid):
        _instance(wl, 0, y0, x0, lam)
    return wl


UNEVEN_SIZES = [(96, 128), (120, 160), (240, 320), (360, 480), (480, 640)]   # (H, W)


def uneven_batch(n_images: int = 64, seeds_per_image: int = 8, n_lambda: int = 16,
                 first_seed: int = 0) -> Workload:
    """64 images of sizes drawn from {128x96, 160x120, 320x240, 480x360, 640x480},
    U{2..8} ellipses, sigma ~ U(0.02, 0.1); 8 random seeds x 16 lambdas in
    [10, 8000] per image.  Image i draws from default_rng(first_seed + i) in the
    order: size, ellipse count, sigma, image, seeds."""
    wl = Workload("uneven-64")
    lam = lambda_schedule(n_lambda, 10, 8000)
    for i in range(n_images):
        rng = np.random.default_rng(first_seed + i)
        H, W = UNEVEN_SIZES[int(rng.integers(0, len(UNEVEN_SIZES)))]
        n_ell = int(rng.integers(2, 9))
        sigma = float(rng.uniform(0.02, 0.1))
        wl.images.append(_image(H, W, n_ell, sigma, rng))
        for _ in range(seeds_per_image):
            y0, x0 = random_seed_origin(H, W, rng)
            _instance(wl, len(wl.images) - 1, y0, x0, lam)
    return wl


@dataclass
class Request:
    arrival_s: float
    workload: Workload


def serving_stream(rate_per_s: float, n_requests: int, seed: int = 0,
                   max_side: int = 800) -> list[Request]:
    """Poisson arrivals; each request is one image with W ~ U{160..max_side}
    step 8, H = 3W/4, U{2..8} ellipses, sigma ~ U(0.02, 0.1), U{4..32} random
    seeds and U{10..30} lambdas in [10, 8000]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        W = int(rng.integers(160 // 8, max_side // 8 + 1)) * 8
        H = 3 * W // 4
        n_ell = int(rng.integers(2, 9))
        sigma = float(rng.uniform(0.02, 0.1))
        n_seeds = int(rng.integers(4, 33))
        n_lam = int(rng.integers(10, 31))
        wl = Workload(f"request-{r}")
        wl.images.append(_image(H, W, n_ell, sigma, rng))
        lam = lambda_schedule(n_lam, 10, 8000)
        for _ in range(n_seeds):
            y0, x0 = random_seed_origin(H, W, rng)
            _instance(wl, 0, y0, x0, lam)
        out.append(Request(t, wl))
    return out


def random_grid(H: int, W: int, rng: np.random.Generator, wmax: int = 20,
                tmax: int = 40, p_zero: float = 0.2, n_lambda: int = 1,
                lam_max: int = 30) -> Workload:
    """A small random grid instance for edge-case tests: random pairwise and
    terminal capacities with a fraction of exact zeros (ties and disconnected
    pieces), a random slope in {0, 1, 2} and a random increasing schedule."""
    def rnd(hi):
        a = rng.integers(0, hi + 1, size=(H, W)).astype(np.int32)
        a[rng.random((H, W)) < p_zero] = 0
        return a
    w_h, w_v = rnd(wmax), rnd(wmax)
    w_h[:, -1] = 0
    w_v[-1, :] = 0
    src0, sink = rnd(tmax), rnd(tmax)
    slope = rng.integers(0, 3, size=(H, W)).astype(np.int32)
    lam = np.sort(rng.choice(np.arange(0, lam_max + 1), size=n_lambda, replace=False)).astype(np.int32)
    wl = Workload(f"random-{H}x{W}")
    wl.images.append(Image(H, W, w_h, w_v, None))
    wl.instances.append(Instance(0, src0, slope, sink, lam))
    return wl
