"""Readers for the paper's worked examples stored beside this file."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def read(name):
    """Returns (body text, {key: [ints]}) of a fixture; '#@ key v...' lines hold values."""
    text = open(os.path.join(HERE, name)).read()
    vals = {}
    for line in text.splitlines():
        if line.startswith("#@"):
            parts = line[2:].split()
            vals[parts[0]] = [int(x) for x in parts[1:]]
    return text, vals
