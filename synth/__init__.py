"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module draws random numbers and lays them out; it holds none of the
processor's arithmetic. Both sides of every parity check receive the arrays it
returns, so neither side has to re-implement the other's generator.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based: draw i of the stream
with key s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15). Uniforms take the top
53 bits; normals use the cosine branch of Box-Muller on two uniforms.

Workload recipe (the paper's ERA-5 / IFS / GFS latents and trained weights are
not available, so seeded stand-ins with the paper's latent shapes are used):
  * latent  x ~ N(0, 1), layout [B, D, H, W, C] (channel last), float32;
  * weights Xavier-uniform U(+-sqrt(6 / (fan_in + fan_out))), float32;
  * biases 0, LayerNorm gamma 1, beta 0 -- or, with ``stress=True``,
    biases and beta ~ U(+-0.1) and gamma ~ 1 + U(+-0.1), so that a dropped
    bias or affine term cannot hide behind zeros.
"""
from __future__ import annotations

import dataclasses
import struct

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# tensor ids inside one block, in file order
BLOCK_TENSORS = ("ln1_g", "ln1_b", "wqkv", "bqkv", "wo", "bo",
                 "ln2_g", "ln2_b", "w1", "b1", "w2", "b2")


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> np.uint64:
    """Key of the sub-stream ``tag`` of ``seed`` (both non-negative ints)."""
    with np.errstate(over="ignore"):
        z = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64) * _GAMMA
        z = z + np.uint64(tag & 0xFFFFFFFFFFFFFFFF)
        return _mix64(z)[0]


def uniform(key: np.uint64, n: int) -> np.ndarray:
    """n draws in [0, 1) as float64."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(np.uint64(key) + i * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(key: np.uint64, n: int) -> np.ndarray:
    """n standard normals (float64), Box-Muller cosine branch."""
    u = uniform(key, 2 * n)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass(frozen=True)
class Shape:
    """Latent grid and processor sizes (level x latitude x longitude x channels)."""
    D: int
    H: int
    W: int
    C: int
    heads: int
    kd: int
    kh: int
    kw: int
    blocks_p6: int = 8
    blocks_p1: int = 4
    lon_periodic: bool = True
    ln_eps: float = 1e-5
    rope: bool = False          # 3D rotary position embedding on q and k

    @property
    def N(self) -> int:
        return self.D * self.H * self.W

    @property
    def block_floats(self) -> int:
        C = self.C
        return 12 * C * C + 13 * C


# 4 x 24 x 48 latent, C=128, 4 heads, window 3x5x5: the small latent.
SMALL = Shape(D=4, H=24, W=48, C=128, heads=4, kd=3, kh=5, kw=5)
# 9 x 90 x 180 latent (2-degree grid, 8 pressure slabs + surface), C=768,
# 16 heads, window 5x7x7: the full-size latent.
FULL = Shape(D=9, H=90, W=180, C=768, heads=16, kd=5, kh=7, kw=7)


def latent(shape: Shape, batch: int, seed: int) -> np.ndarray:
    """[batch, D, H, W, C] float32 latent ~ N(0,1); element b uses sub-stream (seed, b)."""
    out = np.empty((batch, shape.D, shape.H, shape.W, shape.C), dtype=np.float32)
    for b in range(batch):
        key = stream_key(seed, (1 << 40) | b)
        out[b] = normal(key, shape.N * shape.C).reshape(shape.D, shape.H, shape.W, shape.C)
    return out


def _tensor_shapes(C: int):
    return {
        "ln1_g": (C,), "ln1_b": (C,),
        "wqkv": (3 * C, C), "bqkv": (3 * C,),
        "wo": (C, C), "bo": (C,),
        "ln2_g": (C,), "ln2_b": (C,),
        "w1": (4 * C, C), "b1": (4 * C,),
        "w2": (C, 4 * C), "b2": (C,),
    }


def block_weights(C: int, seed: int, proc: int, block: int, stress: bool = False) -> dict:
    """float32 weights of block ``block`` of processor ``proc`` (0 six-hour, 1 one-hour).

    Matrices are [out_features, in_features]; Xavier bounds use those fans.
    """
    shapes = _tensor_shapes(C)
    out = {}
    for tid, name in enumerate(BLOCK_TENSORS):
        shp = shapes[name]
        n = int(np.prod(shp))
        key = stream_key(seed, (2 << 40) | (proc << 24) | (block << 8) | tid)
        if len(shp) == 2:
            fan_out, fan_in = shp
            bound = np.sqrt(6.0 / (fan_in + fan_out))
            vals = (2.0 * uniform(key, n) - 1.0) * bound
        elif name.endswith("_g"):
            vals = 1.0 + (2.0 * uniform(key, n) - 1.0) * 0.1 if stress else np.ones(n)
        else:
            vals = (2.0 * uniform(key, n) - 1.0) * 0.1 if stress else np.zeros(n)
        out[name] = vals.astype(np.float32).reshape(shp)
    return out


def processor_weights(shape: Shape, seed: int, stress: bool = False):
    """(six-hour blocks, one-hour blocks): lists of per-block weight dicts."""
    p6 = [block_weights(shape.C, seed, 0, i, stress) for i in range(shape.blocks_p6)]
    p1 = [block_weights(shape.C, seed, 1, i, stress) for i in range(shape.blocks_p1)]
    return p6, p1


def pack_weights(p6, p1) -> np.ndarray:
    """Flat float32 blob: six-hour blocks then one-hour blocks, tensors in BLOCK_TENSORS order."""
    parts = []
    for blk in list(p6) + list(p1):
        for name in BLOCK_TENSORS:
            parts.append(np.ascontiguousarray(blk[name], dtype=np.float32).ravel())
    return np.concatenate(parts) if parts else np.zeros(0, np.float32)


WEIGHT_MAGIC = b"WM3WGT1\x00"


def write_weight_file(path, shape: Shape, p6, p1) -> None:
    """Weight file: 8-byte magic, int32 C, blocks_p6, blocks_p1, 0, then the packed blob."""
    blob = pack_weights(p6, p1)
    with open(path, "wb") as f:
        f.write(WEIGHT_MAGIC)
        f.write(struct.pack("<4i", shape.C, len(p6), len(p1), 0))
        f.write(blob.astype("<f4").tobytes())


# ----------------------------------------------------------- encoder / decoder

@dataclasses.dataclass(frozen=True)
class Codec:
    """Encoder / decoder sizes: the 0.25-degree grid and the patching into the latent.

    Physical fields: atmosphere [levels, H0, W0, v_atm], surface input
    [H0, W0, v_sfc_in], constants [H0, W0, n_const]; outputs atmosphere
    [levels, H0, W0, v_atm] and surface [H0, W0, v_sfc_out]. The atmosphere is
    zero-padded at the top to level_pad levels; a latent token covers pd
    levels x p x p pixels (atmosphere) or p x p pixels (surface), so the latent
    has level_pad / pd atmospheric levels plus one surface level.
    """
    H0: int
    W0: int
    levels: int = 28
    level_pad: int = 32
    pd: int = 4
    p: int = 8
    v_atm: int = 5
    v_sfc_in: int = 8
    v_sfc_out: int = 17
    n_const: int = 8
    Ce: int = 1024
    heads: int = 16
    kd: int = 5
    kh: int = 7
    kw: int = 7
    blocks: int = 2
    lon_periodic: bool = True
    ln_eps: float = 1e-5

    @property
    def D(self) -> int:
        return self.level_pad // self.pd + 1

    @property
    def H(self) -> int:
        return self.H0 // self.p

    @property
    def W(self) -> int:
        return self.W0 // self.p

    @property
    def k_atm(self) -> int:     # inputs of one atmospheric token
        return self.pd * self.p * self.p * self.v_atm

    @property
    def k_sfc(self) -> int:     # inputs of one surface token
        return self.p * self.p * (self.v_sfc_in + self.n_const)

    @property
    def n_sfc_out(self) -> int:  # outputs of one surface token
        return self.p * self.p * self.v_sfc_out

    def block_shape(self) -> Shape:
        """The NA blocks' shape inside the encoder / decoder (width Ce)."""
        return Shape(D=self.D, H=self.H, W=self.W, C=self.Ce, heads=self.heads, kd=self.kd, kh=self.kh,
                     kw=self.kw, blocks_p6=self.blocks, blocks_p1=self.blocks, lon_periodic=self.lon_periodic,
                     ln_eps=self.ln_eps)


# 0.25-degree grid (720 x 1440, the 721st latitude row dropped), 28 pressure
# levels padded to 32: latent 9 x 90 x 180, encoder / decoder width 1024.
FULL_CODEC = Codec(H0=720, W0=1440)
# 192 x 384 grid, 10 levels padded to 12 (4 per token, 3 atmospheric latent
# levels): latent 4 x 24 x 48
# with the small latent's window and heads, width 128.
SMALL_CODEC = Codec(H0=192, W0=384, levels=10, level_pad=12, pd=4, Ce=128, heads=4, kd=3, kh=5, kw=5)

CODEC_TENSORS = ("embed_atm_w", "embed_atm_b", "embed_sfc_w", "embed_sfc_b", "enc_out_w", "enc_out_b",
                 "dec_in_w", "dec_in_b", "unembed_atm_w", "unembed_atm_b", "unembed_sfc_w", "unembed_sfc_b")


def _codec_shapes(cd: Codec, C: int):
    return {
        "embed_atm_w": (cd.Ce, cd.k_atm), "embed_atm_b": (cd.Ce,),
        "embed_sfc_w": (cd.Ce, cd.k_sfc), "embed_sfc_b": (cd.Ce,),
        "enc_out_w": (C, cd.Ce), "enc_out_b": (C,),
        "dec_in_w": (cd.Ce, C), "dec_in_b": (cd.Ce,),
        "unembed_atm_w": (cd.k_atm, cd.Ce), "unembed_atm_b": (cd.k_atm,),
        "unembed_sfc_w": (cd.n_sfc_out, cd.Ce), "unembed_sfc_b": (cd.n_sfc_out,),
    }


def codec_weights(cd: Codec, C: int, seed: int, stress: bool = False) -> dict:
    """Encoder / decoder weights for a latent of width C (float32).

    Matrices [out, in], Xavier-uniform; biases 0 (U(+-0.1) with stress).
    'enc_blocks' / 'dec_blocks': lists of block weight dicts at width Ce
    (processor ids 2 and 3 of the block generator).
    """
    out = {}
    for tid, (name, shp) in enumerate(_codec_shapes(cd, C).items()):
        n = int(np.prod(shp))
        key = stream_key(seed, (3 << 40) | tid)
        if len(shp) == 2:
            bound = np.sqrt(6.0 / (shp[0] + shp[1]))
            vals = (2.0 * uniform(key, n) - 1.0) * bound
        else:
            vals = (2.0 * uniform(key, n) - 1.0) * 0.1 if stress else np.zeros(n)
        out[name] = vals.astype(np.float32).reshape(shp)
    out["enc_blocks"] = [block_weights(cd.Ce, seed, 2, i, stress) for i in range(cd.blocks)]
    out["dec_blocks"] = [block_weights(cd.Ce, seed, 3, i, stress) for i in range(cd.blocks)]
    return out


def pack_codec_weights(w: dict) -> np.ndarray:
    """Flat float32 blob: CODEC_TENSORS in order, then the encoder blocks and
    the decoder blocks (tensors in BLOCK_TENSORS order)."""
    parts = [np.ascontiguousarray(w[name], dtype=np.float32).ravel() for name in CODEC_TENSORS]
    parts.append(pack_weights(w["enc_blocks"], w["dec_blocks"]))
    return np.concatenate(parts)


def codec_inputs(cd: Codec, seed: int):
    """(atmosphere [levels,H0,W0,v_atm], surface [H0,W0,v_sfc_in], constants [H0,W0,n_const]), float32.

    Fields ~ N(0, 1). Constants in the order of Appendix A.2's list: sin and
    cos of latitude, sin and cos of longitude (cell centres), land-sea mask
    (0/1), soil type (integer class 0..7), topography and elevation (N(0, 1));
    with n_const != 8 the channels after the fourth are N(0, 1).
    """
    atm = normal(stream_key(seed, (4 << 40) | 0), cd.levels * cd.H0 * cd.W0 * cd.v_atm)
    sfc = normal(stream_key(seed, (4 << 40) | 1), cd.H0 * cd.W0 * cd.v_sfc_in)
    const = np.empty((cd.H0, cd.W0, cd.n_const), dtype=np.float64)
    lat = np.deg2rad(90.0 - (np.arange(cd.H0) + 0.5) * 180.0 / cd.H0)
    lon = np.deg2rad((np.arange(cd.W0) + 0.5) * 360.0 / cd.W0)
    base = [np.sin(lat)[:, None] + 0 * lon[None, :], np.cos(lat)[:, None] + 0 * lon[None, :],
            0 * lat[:, None] + np.sin(lon)[None, :], 0 * lat[:, None] + np.cos(lon)[None, :]]
    for c in range(cd.n_const):
        if c < 4:
            const[..., c] = base[c]
        else:
            u = uniform(stream_key(seed, (4 << 40) | (2 + c)), cd.H0 * cd.W0).reshape(cd.H0, cd.W0)
            if c == 4:
                const[..., c] = (u < 0.3).astype(np.float64)
            elif c == 5:
                const[..., c] = np.floor(u * 8.0)
            else:
                const[..., c] = normal(stream_key(seed, (4 << 40) | (2 + c)), cd.H0 * cd.W0).reshape(cd.H0, cd.W0)
    return (atm.reshape(cd.levels, cd.H0, cd.W0, cd.v_atm).astype(np.float32),
            sfc.reshape(cd.H0, cd.W0, cd.v_sfc_in).astype(np.float32),
            const.astype(np.float32))
