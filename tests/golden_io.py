"""Readers for the fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [l.split("#")[0].strip() for l in f if l.split("#")[0].strip()]


def splitmix64():
    return [int(l, 16) for l in lines("splitmix64.txt")]


def he_standard():
    return {int(a): int(b) for a, b in (l.split() for l in lines("he_standard_128.txt"))}


def parameterise():
    out = {}
    for l in lines("parameterise.txt"):
        v = [int(x) for x in l.split()]
        out[v[0]] = (v[1], v[2:])
    return out


def primes():
    out = {}
    for l in lines("primes.txt"):
        n, rest = l.split(":")
        out[int(n)] = [int(x, 16) for x in rest.split()]
    return out


def sigmoid_coeffs():
    return [float(x) for x in lines("sigmoid_approximate.txt")[0].split()]
