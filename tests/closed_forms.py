"""Textbook closed-form view factors, written from the mathematics (test helpers).

* parallel, directly opposed rectangles a x b at distance c;
* parallel rectangles in parallel planes with arbitrary offsets (superposition of
  the corner function G, as tabulated in view-factor catalogues);
* perpendicular rectangles sharing an edge;
* coaxial parallel discs (the thesis's Eq. 6.1-6.2).
"""
import math


def parallel_opposed(a, b, c):
    X, Y = a / c, b / c
    x1, y1 = math.sqrt(1 + X * X), math.sqrt(1 + Y * Y)
    return (2.0 / (math.pi * X * Y)) * (
        math.log(x1 * y1 / math.sqrt(1 + X * X + Y * Y))
        + X * y1 * math.atan(X / y1) + Y * x1 * math.atan(Y / x1)
        - X * math.atan(X) - Y * math.atan(Y))


def _corner_G(x, y, eta, xi, z):
    u, v = x - xi, y - eta
    r1 = math.sqrt(u * u + z * z)
    r2 = math.sqrt(v * v + z * z)
    t1 = v * r1 * math.atan(v / r1) if r1 > 0 else 0.0
    t2 = u * r2 * math.atan(u / r2) if r2 > 0 else 0.0
    s = u * u + v * v + z * z
    t3 = 0.5 * z * z * math.log(s) if s > 0 else 0.0
    return (t1 + t2 - t3) / (2.0 * math.pi)


def parallel_rectangles(x1, x2, y1, y2, xi1, xi2, eta1, eta2, z):
    """F from [x1,x2]x[y1,y2] (plane 0) to [xi1,xi2]x[eta1,eta2] (plane z), facing each other."""
    tot = 0.0
    for i, x in enumerate((x1, x2), 1):
        for j, y in enumerate((y1, y2), 1):
            for k, eta in enumerate((eta1, eta2), 1):
                for l, xi in enumerate((xi1, xi2), 1):
                    tot += (-1) ** (i + j + k + l) * _corner_G(x, y, eta, xi, z)
    return tot / ((x2 - x1) * (y2 - y1))


def perpendicular_common_edge(l, h, w):
    """F from the w x l rectangle to the h x l rectangle sharing the edge of length l."""
    H, W = h / l, w / l
    A = W * math.atan(1 / W) + H * math.atan(1 / H) - math.sqrt(H * H + W * W) * math.atan(1 / math.sqrt(H * H + W * W))
    t1 = (1 + W * W) * (1 + H * H) / (1 + W * W + H * H)
    t2 = (W * W * (1 + W * W + H * H) / ((1 + W * W) * (W * W + H * H))) ** (W * W)
    t3 = (H * H * (1 + H * H + W * W) / ((1 + H * H) * (H * H + W * W))) ** (H * H)
    return (A + 0.25 * math.log(t1 * t2 * t3)) / (math.pi * W)


def coaxial_discs(r1, r2, h):
    """F from disc of radius r1 to the coaxial disc r2 at distance h (Eq. 6.1-6.2)."""
    R1, R2 = r1 / h, r2 / h
    X = 1 + (1 + R2 * R2) / (R1 * R1)
    return 0.5 * (X - math.sqrt(X * X - 4 * (R2 / R1) ** 2))
